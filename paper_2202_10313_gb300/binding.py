"""Python binding of the C ABI in include/ader_lts.h (argument marshalling only).

Every step of the solver runs inside libaderlts.so; this module converts numpy arrays
and torch streams / device memory into the plain pointers the ABI takes. It raises if
the library has not been built: there is no fallback implementation.
"""
import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaderlts.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ader_lts.h")

LTS_OK, LTS_ERR_ARG, LTS_ERR_MESH, LTS_ERR_CUDA, LTS_ERR_OOM, LTS_ERR_STATE, LTS_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
LTS_ERR_NONFINITE = -7
BC_INTERIOR, BC_ABSORBING, BC_FREE_SURFACE, BC_PERIODIC = 0, 1, 2, 3

_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_int64
_D = ctypes.c_double
_SIGS = {
    "lts_create": (_I, [_I, _I, _I, _I, ctypes.POINTER(_P)]),
    "lts_destroy": (None, [_P]),
    "lts_last_error": (ctypes.c_char_p, [_P]),
    "lts_set_mesh": (_I, [_P, _L, _P, _L, _P, _P, _P]),
    "lts_set_material": (_I, [_P, _P, _P, _P, _P, _P, _D, _D]),
    "lts_setup_clusters": (_I, [_P, _I, _D, _D, _P, _P, _P]),
    "lts_force_clusters": (_I, [_P, _I, _P, _D, _D]),
    "lts_state_bytes": (_I, [_P, _I, _P]),
    "lts_bind_device_memory": (_I, [_P, _P, _L]),
    "lts_quadrature_points": (_I, [_P, _P, _P]),
    "lts_project_initial": (_I, [_P, _P]),
    "lts_set_dofs": (_I, [_P, _P]),
    "lts_get_dofs": (_I, [_P, _P]),
    "lts_set_dofs_subset": (_I, [_P, _L, _P, _P]),
    "lts_get_dofs_subset": (_I, [_P, _L, _P, _P]),
    "lts_add_point_source": (_I, [_P, _I, _P, _P, _D, _D, _D]),
    "lts_add_receiver": (_I, [_P, _P, _D, _P]),
    "lts_advance": (_I, [_P, _D, _P]),
    "lts_advance_steps": (_I, [_P, _L, _P]),
    "lts_get_seismogram": (_I, [_P, _I, _I, _P, _P, _L, _P]),
    "lts_energy": (_I, [_P, _P]),
    "lts_info": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "lts_set_profiling": (_I, [_P, _I]),
    "lts_kernel_stats": (_I, [_P, _P, _P, _P]),
    "lts_transfer_bytes": (_I, [_P, _P, _P]),
    "lts_set_contraction": (_I, [_P, _I]),
    "lts_set_tile": (_I, [_P, _I]),
    "lts_launch_config": (_I, [_P, _P, _P]),
    "lts_autotune": (_I, [_P, _I, _P, _P, _P, _P, _I, _P]),
    "lts_set_wait_limit": (_I, [_P, _L, _I]),
    "lts_set_adjoint_memory": (_I, [_P, ctypes.c_uint64]),
    "lts_measure_peaks": (_I, [_P, _P, _P]),
    "lts_adjoint_source_gradient": (_I, [_P, _P]),
    "lts_partition": (_I, [_P, _I, _P, _P]),
    "lts_cut_faces": (_I, [_P, _P, _L, _P, _P]),
    "lts_set_partition": (_I, [_P, _I, _P]),
    "lts_exchange_bytes": (_I, [_P, _P]),
    "lts_set_graphs": (_I, [_P, _I]),
    "lts_checkpoint_save": (_I, [_P, ctypes.c_char_p]),
    "lts_checkpoint_load": (_I, [_P, ctypes.c_char_p]),
    "lts_set_finest_dt": (_I, [_P, _D]),
    "lts_misfit_gradient": (_I, [_P, _L, _L, _P, _P, _P, _P, _P, _P]),
    "lts_energy_noalloc": (_I, [_I, _I, _P, _P, _L, _P, _P]),
    "lts_reference_operators": (_I, [_I, _P, _P, _P]),
    "lts_eval_basis": (_I, [_I, _L, _P, _P]),
    "lts_quadrature_rule": (_I, [_I, _P, _P, _P]),
}


def reference_operators(order):
    """(K (3,B,B), Ft (4,B,F), Fb (4,3,B,F)) from the library's exact integration."""
    B = order * (order + 1) * (order + 2) // 6
    F = order * (order + 1) // 2
    K = np.zeros((3, B, B))
    Ft = np.zeros((4, B, F))
    Fb = np.zeros((4, 3, B, F))
    rc = lib().lts_reference_operators(order, _ptr(K), _ptr(Ft), _ptr(Fb))
    if rc != LTS_OK:
        raise LtsError(rc, "lts_reference_operators")
    return K, Ft, Fb


def eval_basis(order, xi):
    xi = np.ascontiguousarray(np.atleast_2d(xi), dtype=np.float64)
    B = order * (order + 1) * (order + 2) // 6
    out = np.zeros((xi.shape[0], B))
    rc = lib().lts_eval_basis(order, xi.shape[0], _ptr(xi), _ptr(out))
    if rc != LTS_OK:
        raise LtsError(rc, "lts_eval_basis")
    return out


def quadrature_rule(order):
    n = ctypes.c_int64()
    lib().lts_quadrature_rule(order, ctypes.byref(n), None, None)
    xi = np.zeros((n.value, 3))
    w = np.zeros(n.value)
    rc = lib().lts_quadrature_rule(order, ctypes.byref(n), _ptr(xi), _ptr(w))
    if rc != LTS_OK:
        raise LtsError(rc, "lts_quadrature_rule")
    return xi, w


def header_functions():
    """Names of the functions declared in include/ader_lts.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lts_[a-z_0-9]+)\s*\(", text)))


def lib():
    """Load libaderlts.so (built in-tree by paper_2202_10313_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libaderlts.so is not built; run paper_2202_10313_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class LtsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%d: %s" % (code, msg))
        self.code = code


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Solver:
    """One solver handle (lts_t*). Method names follow the C functions."""

    def __init__(self, order, n_mech=0, device=0, n_fused=1):
        """n_fused > 1: fused simulations; DOF arrays then carry a leading simulation axis
        (n_fused, K, n_q, B) and sources / seismograms take a simulation index."""
        self.order, self.n_mech, self.device, self.n_fused = order, n_mech, device, n_fused
        self.n_sources = 0
        self.nq = 9 + 6 * n_mech
        self.nb = order * (order + 1) * (order + 2) // 6
        self._h = ctypes.c_void_p()
        self._mem = None
        rc = lib().lts_create(order, n_mech, n_fused, device, ctypes.byref(self._h))
        if rc != LTS_OK:
            raise LtsError(rc, "lts_create failed")

    def _check(self, rc):
        if rc != LTS_OK:
            msg = lib().lts_last_error(self._h)
            raise LtsError(rc, msg.decode() if msg else "")

    def close(self):
        if self._h:
            lib().lts_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- set-up
    def set_mesh(self, xyz, tet, face_bc, period=None):
        xyz = _f64(xyz)
        tet = np.ascontiguousarray(tet, dtype=np.int64)
        bc = np.ascontiguousarray(face_bc, dtype=np.int32)
        self.K = tet.shape[0]
        per = None if period is None else _f64(period, 3)
        self._check(lib().lts_set_mesh(self._h, xyz.shape[0], _ptr(xyz), self.K, _ptr(tet), _ptr(bc), _ptr(per)))
        self.n_sources = 0   # a new mesh drops the sources

    def set_material(self, rho, vp, vs, qp=None, qs=None, f_min=0.1, f_max=5.0):
        K = self.K
        arrs = [_f64(rho, K), _f64(vp, K), _f64(vs, K)]
        q = [None if x is None else _f64(x, K) for x in (qp, qs)]
        self._check(lib().lts_set_material(self._h, *[_ptr(a) for a in arrs], _ptr(q[0]), _ptr(q[1]),
                                           float(f_min), float(f_max)))

    def add_point_source(self, x, m6, f0, t0, m0=1.0, fused_idx=0):
        self._check(lib().lts_add_point_source(self._h, fused_idx, _ptr(_f64(x, 3)), _ptr(_f64(m6, 6)),
                                               float(f0), float(t0), float(m0)))
        self.n_sources += 1

    def add_receiver(self, x, dt_sample):
        rid = ctypes.c_int()
        self._check(lib().lts_add_receiver(self._h, _ptr(_f64(x, 3)), float(dt_sample), ctypes.byref(rid)))
        return rid.value

    def use_torch_memory(self, n_clusters=1):
        """Allocate the device state through torch and bind it to the handle."""
        import torch
        nbytes = ctypes.c_int64()
        self._check(lib().lts_state_bytes(self._h, n_clusters, ctypes.byref(nbytes)))
        t = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda:%d" % self.device)
        base = t.data_ptr()
        off = (-base) % 256
        self._check(lib().lts_bind_device_memory(self._h, ctypes.c_void_p(base + off), nbytes.value))
        self._mem = t

    def setup_clusters(self, n_clusters, cfl, lam=None):
        cl = np.zeros(self.K, dtype=np.int32)
        lam_out, sp = ctypes.c_double(), ctypes.c_double()
        self._check(lib().lts_setup_clusters(self._h, n_clusters, float(cfl), -1.0 if lam is None else float(lam),
                                             _ptr(cl), ctypes.byref(lam_out), ctypes.byref(sp)))
        return cl, lam_out.value, sp.value

    def force_clusters(self, clusters, n_clusters, cfl, lam=1.0):
        cl = np.ascontiguousarray(clusters, dtype=np.int32)
        self._check(lib().lts_force_clusters(self._h, n_clusters, _ptr(cl), float(cfl), float(lam)))

    # ----------------------------------------------------------------- state
    def quadrature_points(self):
        n = ctypes.c_int64()
        self._check(lib().lts_quadrature_points(self._h, ctypes.byref(n), None))
        out = np.zeros((self.K, n.value, 3))
        self._check(lib().lts_quadrature_points(self._h, ctypes.byref(n), _ptr(out)))
        return out

    def project_initial(self, fn):
        pts = self.quadrature_points()
        vals = np.ascontiguousarray(np.asarray(fn(pts.reshape(-1, 3)), dtype=np.float64).reshape(
            pts.shape[0], pts.shape[1], self.nq))
        self._check(lib().lts_project_initial(self._h, _ptr(vals)))

    def _dof_shape(self, n):
        return (n, self.nq, self.nb) if self.n_fused == 1 else (self.n_fused, n, self.nq, self.nb)

    def set_dofs(self, dofs):
        self._check(lib().lts_set_dofs(self._h, _ptr(_f64(dofs, self.n_fused * self.K * self.nq * self.nb))))

    def get_dofs(self):
        out = np.zeros(self._dof_shape(self.K))
        self._check(lib().lts_get_dofs(self._h, _ptr(out)))
        return out

    def set_dofs_subset(self, elems, dofs):
        el = np.ascontiguousarray(elems, dtype=np.int64)
        d = _f64(dofs, self.n_fused * len(el) * self.nq * self.nb)
        self._check(lib().lts_set_dofs_subset(self._h, len(el), _ptr(el), _ptr(d)))

    def get_dofs_subset(self, elems):
        el = np.ascontiguousarray(elems, dtype=np.int64)
        out = np.zeros(self._dof_shape(len(el)))
        self._check(lib().lts_get_dofs_subset(self._h, len(el), _ptr(el), _ptr(out)))
        return out

    # --------------------------------------------------------------- running
    def advance_steps(self, n_finest, stream=None):
        self._check(lib().lts_advance_steps(self._h, int(n_finest), _stream_handle(stream)))

    def advance(self, t_end, stream=None):
        self._check(lib().lts_advance(self._h, float(t_end), _stream_handle(stream)))

    def seismogram(self, rid, fused_idx=0):
        n = ctypes.c_int64()
        self._check(lib().lts_get_seismogram(self._h, rid, fused_idx, None, None, 0, ctypes.byref(n)))
        t = np.zeros(n.value)
        v = np.zeros((n.value, 9))
        self._check(lib().lts_get_seismogram(self._h, rid, fused_idx, _ptr(t), _ptr(v), n.value, ctypes.byref(n)))
        return t, v

    def energy(self):
        e = ctypes.c_double()
        self._check(lib().lts_energy(self._h, ctypes.byref(e)))
        return e.value

    def info(self):
        nc = ctypes.c_int()
        ce = np.zeros(8, dtype=np.int64)
        up = np.zeros(8, dtype=np.int64)
        dtm, lam, fdt, tn = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        nl = ctypes.c_int64()
        self._check(lib().lts_info(self._h, ctypes.byref(nc), _ptr(ce), _ptr(up), ctypes.byref(dtm), ctypes.byref(lam),
                                   ctypes.byref(fdt), ctypes.byref(tn), ctypes.byref(nl)))
        n = nc.value
        return dict(n_clusters=n, cluster_elems=ce[:n].copy(), updates_per_macro=up[:n].copy(), dt_min=dtm.value,
                    lam=lam.value, finest_dt=fdt.value, time=tn.value, launches=nl.value)

    def transfer_bytes(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(lib().lts_transfer_bytes(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def launch_config(self):
        """Resident CTAs per SM and threads per CTA of (predict, neighbour, predict on tensor cores)."""
        c = np.zeros(3, dtype=np.int32)
        t = np.zeros(3, dtype=np.int32)
        self._check(lib().lts_launch_config(self._h, _ptr(c), _ptr(t)))
        return dict(ctas_per_sm=c.tolist(), threads=t.tolist())

    def autotune(self, allow_tf32=False, stream=None):
        """Time the candidate launch configurations on a snapshot of the state and keep the
        fastest; returns the choice and every candidate's milliseconds per macro step."""
        chosen = np.zeros(4, dtype=np.int32)
        best = ctypes.c_double()
        table = np.zeros((32, 5))
        n = ctypes.c_int()
        self._check(lib().lts_autotune(self._h, 1 if allow_tf32 else 0, _stream_handle(stream), _ptr(chosen),
                                       ctypes.byref(best), _ptr(table), 32, ctypes.byref(n)))
        names = {0: "fp32", 1: "tf32x3", 2: "tf32", 3: "sparse"}
        rows = [dict(contraction=names[int(r[0])], ctas_predict=int(r[1]), ctas_neighbour=int(r[2]), tile=int(r[3]),
                     ms=float(r[4])) for r in table[:min(n.value, 32)]]
        return dict(contraction=names[int(chosen[0])], ctas_predict=int(chosen[1]), ctas_neighbour=int(chosen[2]),
                    tile=int(chosen[3]), best_ms=best.value, candidates=rows)

    def partition(self, n_parts):
        """Weighted partition (part per element) and its statistics."""
        part = np.zeros(self.K, dtype=np.int32)
        st = np.zeros(6)
        self._check(lib().lts_partition(self._h, int(n_parts), _ptr(part), _ptr(st)))
        keys = ("max_load", "min_load", "total_weight", "cut_faces", "msgs_per_macro", "buffer_msgs_per_macro")
        return part, dict(zip(keys, st.tolist()))

    def cut_faces(self, part):
        """Exchange plan: rows (recv elem, recv face, send elem, send face, orient, recv part,
        send part, recv cluster) in message order."""
        p = np.ascontiguousarray(part, dtype=np.int32)
        n = ctypes.c_int64()
        self._check(lib().lts_cut_faces(self._h, _ptr(p), 0, None, ctypes.byref(n)))
        out = np.zeros((n.value, 8), dtype=np.int64)
        self._check(lib().lts_cut_faces(self._h, _ptr(p), n.value, _ptr(out), ctypes.byref(n)))
        return out

    def set_partition(self, part=None, n_parts=None):
        if part is None:
            self._check(lib().lts_set_partition(self._h, 1, None))
            return
        p = np.ascontiguousarray(part, dtype=np.int32)
        self._check(lib().lts_set_partition(self._h, int(n_parts if n_parts else p.max() + 1), _ptr(p)))

    def exchange_bytes(self):
        b = ctypes.c_int64()
        self._check(lib().lts_exchange_bytes(self._h, ctypes.byref(b)))
        return b.value

    def set_finest_dt(self, dt):
        self._check(lib().lts_set_finest_dt(self._h, float(dt)))

    def misfit_gradient(self, n_steps, data, every=100, stream=None, want_dq0=False, want_grad=True):
        """J, dJ/d(rho, lambda, mu) (K, 3), synthetic samples (shape of data: one row per
        sample time, then n_rec, 3; fused: sample time, F, n_rec, 3) and optionally dJ/dQ at the
        start ((K, 9, B); fused (F, K, 9, B)), by the discrete adjoint of the time loop (GTS:
        samples every step; LTS: every macro step). Fused runs give J and the gradient summed
        over the simulations."""
        data = np.ascontiguousarray(data, dtype=np.float64)
        J = ctypes.c_double()
        grad = np.zeros((self.K, 3))
        syn = np.zeros(data.shape)
        shape = (self.K, 9, self.nb) if self.n_fused == 1 else (self.n_fused, self.K, 9, self.nb)
        dq0 = np.zeros(shape) if want_dq0 else None
        self._check(lib().lts_misfit_gradient(self._h, int(n_steps), int(every), _ptr(data), ctypes.byref(J),
                                              _ptr(grad) if want_grad else None, _ptr(syn), _ptr(dq0),
                                              _stream_handle(stream)))
        return (J.value, grad, syn, dq0) if want_dq0 else (J.value, grad, syn)

    def misfit(self, n_steps, data, every=100, stream=None):
        """Forward sweep only: J and the samples."""
        data = np.ascontiguousarray(data, dtype=np.float64)
        J = ctypes.c_double()
        syn = np.zeros(data.shape)
        self._check(lib().lts_misfit_gradient(self._h, int(n_steps), int(every), _ptr(data), ctypes.byref(J), None,
                                              _ptr(syn), None, _stream_handle(stream)))
        return J.value, syn

    def checkpoint_save(self, path):
        self._check(lib().lts_checkpoint_save(self._h, str(path).encode()))

    def checkpoint_load(self, path):
        self._check(lib().lts_checkpoint_load(self._h, str(path).encode()))

    def set_graphs(self, enable=True):
        self._check(lib().lts_set_graphs(self._h, 1 if enable else 0))

    def source_gradient(self):
        """dJ/dm6 (n_sources, 6) of the point sources from the last misfit_gradient call."""
        out = np.zeros((self.n_sources, 6))
        self._check(lib().lts_adjoint_source_gradient(self._h, _ptr(out)))
        return out

    def measure_peaks(self, stream=None):
        """Throughput probes: dict(fp32_tflops, tf32_tflops, fp32_ms, tf32_ms)."""
        out = (ctypes.c_double * 4)()
        self._check(lib().lts_measure_peaks(self._h, _stream_handle(stream), out))
        return dict(fp32_tflops=out[0], tf32_tflops=out[1], fp32_ms=out[2], tf32_ms=out[3])

    def set_adjoint_memory(self, nbytes=0):
        """Budget for the phase inputs the LTS adjoint keeps per checkpoint segment (0: half
        the free device memory)."""
        self._check(lib().lts_set_adjoint_memory(self._h, int(nbytes)))

    def set_wait_limit(self, cycles=2000000000, suppress_commit=False):
        self._check(lib().lts_set_wait_limit(self._h, int(cycles), 1 if suppress_commit else 0))

    def set_contraction(self, mode):
        """'fp32' (CUDA cores), 'sparse' (CUDA cores, generated sparse products), 'tf32x3'
        (tensor cores, split tf32) or 'tf32' (tensor cores)."""
        code = {"fp32": 0, "tf32x3": 1, "tf32": 2, "sparse": 3}[mode]
        self._check(lib().lts_set_contraction(self._h, code))

    def set_tile(self, tile):
        """Tile variant of the sparse engine's neighbour kernel: 0 (8 elements per CTA) or 1 (4, the
        default)."""
        self._check(lib().lts_set_tile(self._h, int(tile)))

    def set_profiling(self, on=True):
        self._check(lib().lts_set_profiling(self._h, 1 if on else 0))

    def kernel_stats(self):
        ms = np.zeros(2)
        nl = np.zeros(2, dtype=np.int64)
        ne = np.zeros(2, dtype=np.int64)
        self._check(lib().lts_kernel_stats(self._h, _ptr(ms), _ptr(nl), _ptr(ne)))
        return dict(ms=ms, launches=nl, elems=ne)
