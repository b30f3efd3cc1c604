/*
 * ader_lts.h -- C ABI of the GB300 ADER-DG solver with clustered local time stepping.
 *
 * Method: "Next-Generation Local Time Stepping for the ADER-DG Finite Element Method"
 * (Breuer & Heinecke). The library advances the 3D elastic (n_mech = 0) or anelastic
 * (n_mech relaxation mechanisms) wave equations, Eq. (1) of Sec. III, on unstructured
 * tetrahedra with the ADER-DG time, volume and surface kernels of Sec. III-A, driven by
 * the rate-2 clustered LTS scheme with buffers B1/B2/B3 of Sec. V. All bulk arithmetic
 * runs in FP32 in CUDA kernels; set-up runs in FP64 on the host.
 *
 * Conventions shared by every call
 *  - Every function returns an int status: LTS_OK (0) or a negative LTS_ERR_* code.
 *    No C++ exception crosses this boundary. lts_last_error() describes the last
 *    failure on a handle (the string stays valid until the next call on it).
 *  - Host arrays are owned by the caller; the library copies what it needs before
 *    returning. Nothing is retained by pointer except the device block given to
 *    lts_bind_device_memory (caller-owned, must outlive the handle's use of it).
 *  - Elements are identified by their index in the caller's tetrahedron array
 *    (original order); the library's internal reordering is never visible.
 *  - Reference tetrahedron v0=(0,0,0), v1=(1,0,0), v2=(0,1,0), v3=(0,0,1); face i of a
 *    tetrahedron (t0,t1,t2,t3) is the vertex triple {(t0,t2,t1), (t0,t1,t3), (t0,t3,t2),
 *    (t1,t2,t3)}[i], i.e. the face opposite local vertex 3-i.
 *  - Quantities per element (rows): sxx, syy, szz, sxy, syz, sxz, u, v, w, then 6
 *    memory variables (xx, yy, zz, xy, yz, xz) per relaxation mechanism.
 *  - DOFs are coefficients of the orthonormal modal (Dubiner) basis of Sec. III-A:
 *    mode (i,j,k) = [s1^i P_i(a)] [s2^j P_j^(2i+1,0)(b)] P_k^(2i+2j+2,0)(c) with
 *    s1 = 1-x2-x3, s2 = 1-x3, a = 2x1/s1-1, b = 2x2/s2-1, c = 2x3-1, unit L2 norm on the
 *    reference tetrahedron; modes ordered by degree i+j+k, then k, then j.
 *    DOF arrays are [element][quantity][mode], row-major, double.
 */
#ifndef ADER_LTS_H
#define ADER_LTS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lts_solver lts_t;

enum {
    LTS_OK = 0,
    LTS_ERR_ARG = -1,      /* invalid argument or unsupported configuration            */
    LTS_ERR_MESH = -2,     /* invalid mesh (orientation, non-conforming or open faces)   */
    LTS_ERR_CUDA = -3,     /* a CUDA runtime call failed                                */
    LTS_ERR_OOM = -4,      /* host or device allocation failed / bound block too small  */
    LTS_ERR_STATE = -5,    /* call out of order (e.g. advance before cluster set-up)   */
    LTS_ERR_TIMEOUT = -6,  /* a bounded device-side wait gave up                       */
    LTS_ERR_NONFINITE = -7 /* a reduction found NaN or Inf in the state                 */
};

/* Fused simulations (Sec. IV-A): n_fused is 1 or a multiple of LTS_FUSED_MULTIPLE up to
 * LTS_MAX_FUSED. */
#define LTS_FUSED_MULTIPLE 4
#define LTS_MAX_FUSED 64

/* Face boundary codes (per tetrahedron face). */
enum { LTS_BC_INTERIOR = 0, LTS_BC_ABSORBING = 1, LTS_BC_FREE_SURFACE = 2, LTS_BC_PERIODIC = 3 };

/* Create a solver. order O in {3,4,5} (B(O) = O(O+1)(O+2)/6 modes, Sec. III-A);
 * n_mech in {0, 3} (N^q = 9 + 6 n_mech quantities, Sec. III); n_fused simulations
 * share mesh, material and clusters and differ in their sources and initial DOFs (fused
 * simulations, Sec. IV-A: every scalar DOF becomes a vector of n_fused values; on the
 * device the simulation index is the innermost one, Q[k][q][b][f]).
 * Selects CUDA device `device` for all later calls on the handle. device < 0 creates a
 * host-only handle: mesh, material and cluster set-up run (lts_setup_clusters reports
 * clusters, lambda and speedup) but no device state exists, so calls that need it
 * return LTS_ERR_STATE. *out is set only on success. Errors: LTS_ERR_ARG, LTS_ERR_CUDA,
 * LTS_ERR_OOM. */
int lts_create(int order, int n_mech, int n_fused, int device, lts_t** out);

/* Release the handle, its device memory (unless caller-bound) and host tables. NULL is a no-op. */
void lts_destroy(lts_t* h);

/* Message describing the last error on h (empty string if none). */
const char* lts_last_error(lts_t* h);

/* Mesh (Sec. III-A: conforming unstructured tetrahedra). xyz[3*n_vert] coordinates,
 * tet[4*n_tet] vertex ids (each tetrahedron positively oriented), face_bc[4*n_tet]
 * LTS_BC_* per face (interior faces 0). period[3] box lengths for periodic faces
 * (matched by vertex position modulo the box), NULL if none. Errors: LTS_ERR_MESH for
 * non-positive orientation, faces shared by != 2 elements, inconsistent orientation or
 * an interior/periodic face without partner; LTS_ERR_ARG for bad sizes or codes. */
int lts_set_mesh(lts_t* h, int64_t n_vert, const double* xyz, int64_t n_tet, const int64_t* tet,
                 const int32_t* face_bc, const double* period);

/* Material per element (Sec. VII-B lists rho, vp, vs, Qp, Qs): unrelaxed velocities.
 * qp/qs are required when n_mech > 0 (constant-Q fit over [f_min, f_max] Hz with
 * log-spaced relaxation frequencies, collocated at those frequencies), ignored
 * otherwise. Errors: LTS_ERR_ARG (non-positive values, missing Q), LTS_ERR_STATE (no mesh). */
int lts_set_material(lts_t* h, const double* rho, const double* vp, const double* vs,
                     const double* qp, const double* qs, double f_min, double f_max);

/* Cluster set-up (Sec. V-A). dt_k = cfl * d_k / ((2O-1) vp_k), d_k the insphere
 * diameter; clusters C_l = [2^(l-1) lam dt_min, 2^l lam dt_min), last open-ended;
 * normalised so face neighbours differ by at most one cluster. lambda <= 0 searches
 * lambda in {0.51, ..., 1.00} (steps of 0.01, ties to the larger) maximising the
 * theoretical speedup. n_clusters = 1 is global time stepping. Outputs (each may be
 * NULL): cluster_out[n_tet] (0-based), lambda_out, speedup_out (GTS cost / LTS cost).
 * Allocates and uploads all device state; resets time to 0 and DOFs to zero.
 * Errors: LTS_ERR_ARG, LTS_ERR_STATE (no material), LTS_ERR_CUDA, LTS_ERR_OOM. */
int lts_setup_clusters(lts_t* h, int n_clusters, double cfl, double lambda,
                       int32_t* cluster_out, double* lambda_out, double* speedup_out);

/* As lts_setup_clusters, with the cluster of every element given (0-based, normalised
 * by the caller) and lambda fixed (1.0 if <= 0). Errors additionally: LTS_ERR_ARG if
 * face neighbours differ by more than one cluster. */
int lts_force_clusters(lts_t* h, int n_clusters, const int32_t* clusters, double cfl, double lambda);

/* Device bytes the state needs after cluster set-up would allocate it; call after
 * lts_set_material. The caller may then hand a block of at least that size (256-byte
 * aligned) to lts_bind_device_memory before lts_setup_clusters; otherwise the library
 * allocates its own block. Errors: LTS_ERR_STATE. */
int lts_state_bytes(lts_t* h, int n_clusters, int64_t* bytes);
int lts_bind_device_memory(lts_t* h, void* dev, int64_t bytes);

/* Physical quadrature points of the projection rule: n_per_elem points per element,
 * xyz_out[n_tet][n_per_elem][3] (NULL to query the count only). */
int lts_quadrature_points(lts_t* h, int64_t* n_per_elem, double* xyz_out);

/* L2 projection of point values: values[n_tet][n_per_elem][n_q] at the points of
 * lts_quadrature_points become the DOFs (orthonormal basis, Sec. III-A) of every
 * fused simulation. */
int lts_project_initial(lts_t* h, const double* values);

/* Raw DOFs [n_fused][n_tet][n_q][B], simulation-major (double on the host, FP32 on the
 * device). lts_get_dofs synchronises the solver's stream. */
int lts_set_dofs(lts_t* h, const double* dofs);
int lts_get_dofs(lts_t* h, double* dofs);

/* DOFs of a subset of elements: elems[n] (original indices), dofs[n_fused][n][n_q][B]
 * in the order of elems. Setting leaves every other element unchanged. Both synchronise the
 * device. Errors: LTS_ERR_STATE before cluster set-up, LTS_ERR_ARG for an index out of
 * range or NULL arrays with n > 0. */
int lts_set_dofs_subset(lts_t* h, int64_t n, const int64_t* elems, const double* dofs);
int lts_get_dofs_subset(lts_t* h, int64_t n, const int64_t* elems, double* dofs);

/* Moment-tensor point source (reading of Sec. VII-B's point sources): moment rate
 * m0 * m6 * s(t), s the Ricker wavelet (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2),
 * m6 = (xx, yy, zz, xy, yz, xz). The containing element (lowest index whose closed
 * tetrahedron holds x) gains -m0 m6 (int s dt) phi_b(xi)/|det J| on its stress DOFs at
 * the end of each of its steps (O-point Gauss-Legendre in time), in simulation fused_idx
 * only (0 <= fused_idx < n_fused). Errors: LTS_ERR_ARG (point outside the mesh, bad
 * fused_idx). Call before lts_setup_clusters. */
int lts_add_point_source(lts_t* h, int fused_idx, const double x[3], const double m6[6],
                         double f0, double t0, double m0);

/* Receiver at x sampled every dt_sample seconds (t_j = j dt_sample): each sample inside a
 * step [t_n, t_n + dt) of the receiver's element is the Taylor series
 * sum_d (t_j - t_n)^d / d! d^dQ evaluated at x (9 elastic quantities), recorded for every
 * fused simulation. *id receives its index. Errors: LTS_ERR_ARG (outside mesh). Call
 * before lts_setup_clusters. */
int lts_add_receiver(lts_t* h, const double x[3], double dt_sample, int* id);

/* Advance whole macro steps (2^(N_c-1) finest steps of lam*dt_min each) until the time is
 * the largest multiple of the macro step not above t_end (plus a 1e-9 relative slack),
 * asynchronously on `cuda_stream` (a cudaStream_t; NULL = legacy default stream). */
int lts_advance(lts_t* h, double t_end, void* cuda_stream);

/* Advance n_finest finest steps (a multiple of 2^(N_c-1)) on `cuda_stream`. */
int lts_advance_steps(lts_t* h, int64_t n_finest, void* cuda_stream);

/* Copy receiver `id`'s samples so far in simulation fused_idx: t_out[n] times and
 * v_out[n][9] values (either may be NULL); *n receives the number of samples (at most cap
 * are written). Synchronises. Errors: LTS_ERR_ARG (bad id or fused_idx). */
int lts_get_seismogram(lts_t* h, int id, int fused_idx, double* t_out, double* v_out,
                       int64_t cap, int64_t* n);

/* Discrete elastic energy sum_k |det J_k| sum_b (rho |v_b|^2/2 + sigma_b : C^-1 sigma_b / 2),
 * summed over the fused simulations, reduced in FP64 on the device. Synchronises. The
 * reduction is also the state's sentinel: a NaN or Inf anywhere in the stresses or
 * velocities makes it non-finite, and the call then stores the value and returns
 * LTS_ERR_NONFINITE. */
int lts_energy(lts_t* h, double* e);

/* Run information. n_clusters_out; per cluster (arrays of length >= 8, may be NULL):
 * elements, and element updates per macro step; dt_min; lambda; finest step; current
 * time; kernel launches issued so far. */
int lts_info(lts_t* h, int* n_clusters_out, int64_t* cluster_elems, int64_t* updates_per_macro,
             double* dt_min, double* lambda, double* finest_dt, double* time_now, int64_t* launches);

/* Kernel timing. With profiling enabled, every predict+local and neighbour launch is
 * bracketed by CUDA events recorded on the launch stream (no synchronisation).
 * lts_kernel_stats synchronises on the last event and returns, per kind (index 0
 * predict+local, 1 neighbour), the summed milliseconds, the number of launches and the
 * elements processed since profiling was enabled or last read; reading resets them. */
int lts_set_profiling(lts_t* h, int enable);
int lts_kernel_stats(lts_t* h, double* ms_out2, int64_t* launches_out2, int64_t* elems_out2);

/* Cumulative bytes the library copied host->device in lts_advance / lts_advance_steps
 * (source and receiver schedules) and device->host in lts_get_seismogram. */
int lts_transfer_bytes(lts_t* h, int64_t* h2d, int64_t* d2h);

/* Contraction engine of the time and volume kernels (Sec. IV: the products of the DOFs
 * with the stiffness matrices K_c). LTS_CONTRACT_FP32: FP32 CUDA cores, dense degree
 * blocks (the paper's block sparsity).
 * LTS_CONTRACT_TF32X3: 5th-generation tensor cores, every operand split into two tf32
 * parts and the three leading products accumulated in FP32 (FP32-level accuracy).
 * LTS_CONTRACT_TF32: tensor cores on the rounded tf32 parts only (about 1e-3 relative
 * error per product). LTS_CONTRACT_SPARSE (the default): FP32 CUDA cores with
 * the products of K_c, of the face matrices F~_i and of their transposes generated at build
 * time from the nonzero entries only (Sec. IV-A "all sparsity"), in the predict kernel and
 * in a neighbour kernel that forms X F-_{j,h} as (X F~_j) R_h (R_h the face-basis map of the
 * orientation); with fused simulations it runs (element, simulation) slots, and a
 * partitioned run keeps the other engines' neighbour kernel. The adjoint's reverse predict
 * pass (lts_misfit_gradient) uses the same generated products (their transposed forms);
 * every other engine takes its dense-block kernel. The tensor-core engines' surface products run on CUDA cores. Takes effect at the next lts_advance. Errors: LTS_ERR_ARG for an unknown mode or a
 * mode the handle's shape has no kernel for (tensor cores: order 3 with one simulation).
 * A tensor-core wait that gives up (bounded, about one second)
 * makes the next synchronising call return LTS_ERR_TIMEOUT. */
enum { LTS_CONTRACT_FP32 = 0, LTS_CONTRACT_TF32X3 = 1, LTS_CONTRACT_TF32 = 2, LTS_CONTRACT_SPARSE = 3 };
int lts_set_contraction(lts_t* h, int mode);

/* Tile variant of the sparse engine's neighbour kernel (Sec. III-A neighbour surface
 * kernel): 0 = 8 elements per CTA (two CTAs per SM), 1 = 4 elements per CTA (four CTAs per
 * SM; the default). The arithmetic per element is the same, so the results are bitwise
 * identical; only the grouping of elements into CTAs changes. Set by lts_autotune; ignored
 * by the other engines. Errors: LTS_ERR_ARG for another value. */
int lts_set_tile(lts_t* h, int tile);

/* Weighted partitioning for distributed runs (Sec. V-C). Element weight 2^(N_c-1-l) (its
 * updates per macro step, cluster l 0-based); face weight = messages per macro step over
 * the face. Recursive coordinate bisection of the centroids at the weighted median, then a
 * greedy boundary pass that lowers the face-weighted cut within a 3 % load tolerance.
 * Needs clusters (lts_setup_clusters; host-only handles work). part_out[n_tet] in
 * [0, n_parts); stats_out[6] = (largest part weight / mean, smallest / mean, total weight,
 * cut faces counted per receiving side, face-local messages per macro step, whole-buffer
 * messages per macro step of the uncompressed scheme: one 9 x B buffer per sending element,
 * receiving part and receiver step). Either output may be NULL. Errors: LTS_ERR_STATE,
 * LTS_ERR_ARG (n_parts < 1 or > n_tet). */
int lts_partition(lts_t* h, int n_parts, int32_t* part_out, double* stats_out);

/* The exchange plan of a partition: every face whose two elements lie in different parts,
 * from the receiving side, in message order (receiving part, sending part, receiver
 * cluster, receiver element, face). faces[cap][8] = (receiving element, its face i, sending
 * element, its face j, orientation h, receiving part, sending part, receiver cluster), all
 * original indices; the sender computes H = X F-_{j,h} (9 x F values) from its buffer X and
 * the receiver applies the flux of face i to it. *n receives the count. */
int lts_cut_faces(lts_t* h, const int32_t* part, int64_t cap, int64_t* faces, int64_t* n);

/* Emulated partitioned run on one device (Sec. V-C): with n_parts > 1 every cut face takes
 * its neighbour contribution from a face-local message instead of the neighbour's buffer —
 * before each neighbour pass a pack kernel computes, on the sending side, H = X F-_{j,h}
 * for the cut faces whose receivers are active, and the receiver's neighbour kernel reads
 * it. The arithmetic is the one of the unpartitioned run, in the same order. Fused runs
 * send one message per simulation. If clusters are set up, re-creates the device state
 * (time 0, DOFs zero). n_parts <= 1 (part may be NULL) switches it off. Errors: LTS_ERR_ARG, LTS_ERR_STATE. */
int lts_set_partition(lts_t* h, int n_parts, const int32_t* part);

/* Face-local message bytes the partitioned run has produced so far (9 x F FP32 values per
 * active cut face, simulation and neighbour pass). */
int lts_exchange_bytes(lts_t* h, int64_t* bytes);

/* Overrides the finest time step (after cluster set-up) with dt seconds, e.g. to hold the
 * step fixed while the material changes (the adjoint's finite-difference checks). The
 * caller is responsible for stability. Errors: LTS_ERR_STATE, LTS_ERR_ARG (dt <= 0). */
int lts_set_finest_dt(lts_t* h, double dt);

/* Discrete adjoint of the time-stepping loop (the misfit objective of Sec. VII-B,
 * summed): from the current state, advances n_steps steps of the elastic scheme (the same
 * launches as lts_advance_steps, sources included) and evaluates
 *   J = 1/2 sum_{m=0..M} sum_r sum_q (v_q(x_r, t_m) - data[m][r][q])^2,
 * v the particle velocity (u, v, w) at receiver r (the handle's receivers, in order)
 * sampled at the macro-step boundaries t_m (every step with one cluster). The reverse
 * sweep applies the transposed time, volume, local and neighbour surface operators phase
 * by phase, recomputing the forward states from checkpoints stored every `every` macro
 * steps, and
 * correlates the adjoint with the forward states; the correlations are contracted with
 * the exact derivatives (forward-mode dual numbers) of the star matrices and the face
 * flux solvers with respect to each element's rho, lambda, mu — the face terms also
 * with respect to the neighbour's. Outputs (each may be NULL except data): *misfit J,
 * grad[n_tet][3] = dJ/d(rho, lambda, mu) per element (original order), synth_out[M+1][n_rec][3]
 * the samples, dq0[n_tet][9][B] = dJ/dQ at the start. The time step is held fixed. The
 * state ends at t_N (as after lts_advance_steps). Needs n_mech = 0 and at least one
 * receiver; a partitioned run (lts_set_partition) gives bitwise the unpartitioned result. Fused simulations (n_fused = F > 1: each its own sources and initial state,
 * the material shared): data and synth_out [..][F][n_rec][3] (simulation before receiver),
 * dq0[F][n_tet][9][B], and J and grad summed over the simulations — the gradient of the
 * summed misfit, as for several sources of one inversion. The sweep is the phase-level
 * one of clustered LTS for every cluster count. Time is counted in macro steps of 2^(N_c-1) finest steps
 * (one cluster, global time stepping: every step): n_steps is a multiple of the macro
 * step, the samples are taken at the macro-step boundaries (data[M+1][n_rec][3],
 * M = n_steps / 2^(N_c-1)), Q is checkpointed every `every` macro steps
 * (ceil(M/every) + 1 copies of Q plus the per-element operators), and the reverse
 * sweep takes the LTS phases backwards over the state (Q, B1, B2, B3): a neighbour pass
 * sends its transposed flux to the adjoint of the buffer it read (B1, B3, B2 or
 * B1 - B2), a predict pass collects the adjoints of the buffers it wrote. The reverse
 * of a phase reads the phase's inputs: Q of its active elements (predict) or B1, B2, B3
 * of the buffer owners (neighbour), kept while the segment from its checkpoint is
 * replayed. When one segment's worth (every x the bytes of one macro step's phase inputs)
 * fits the adjoint memory budget (lts_set_adjoint_memory; default half the free device
 * memory) the segment is replayed once; otherwise its macro-boundary states are kept and
 * each macro step is replayed once more just before its reverse, keeping one macro step's
 * phase inputs. Both orders give bitwise the same results.
 * With grad and dq0 both NULL only the forward sweep and the misfit run.
 * Errors: LTS_ERR_ARG, LTS_ERR_STATE, LTS_ERR_OOM, LTS_ERR_CUDA. */
int lts_misfit_gradient(lts_t* h, int64_t n_steps, int64_t every, const double* data, double* misfit,
                        double* grad, double* synth_out, double* dq0, void* cuda_stream);

/* Moment-tensor gradient from the last lts_misfit_gradient call that ran the reverse sweep
 * (grad or dq0 requested): out[n_src][6] = dJ/dm6 of every point source (registration order,
 * the six components as given to lts_add_point_source; the source time function and m0
 * held fixed). Each neighbour pass that added a source contributes
 * -m0 (int s dt) / |det J| sum_b lambda_Q[elem][r][b] phi_b(xi_s), lambda_Q the adjoint of Q
 * after the pass. Errors: LTS_ERR_ARG (out NULL), LTS_ERR_STATE (no such sweep since the
 * sources last changed). */
int lts_adjoint_source_gradient(lts_t* h, double* out);

/* Throughput probes of the GPU the handle runs on, for roofline denominators: FP32 FMA on
 * the CUDA cores (8 independent FMA chains per thread, 8 CTAs of 256 threads per SM) and
 * tcgen05 MMA of kind tf32 (M = 128, N = 256, K = 8, FP32 accumulation in tensor memory,
 * one CTA per SM issuing back-to-back products). Each is timed with CUDA events on
 * `cuda_stream` after one warm-up launch. out[4] = FP32 TFLOP/s, tf32 TFLOP/s, and the two
 * timed durations in ms. Synchronises the stream. Errors: LTS_ERR_ARG (out NULL),
 * LTS_ERR_TIMEOUT (a tensor-core wait ran out; its tensor memory is released),
 * LTS_ERR_CUDA. */
int lts_measure_peaks(lts_t* h, void* cuda_stream, double* out);

/* Device-memory budget in bytes for the phase inputs the LTS adjoint keeps per segment
 * (see lts_misfit_gradient); 0 restores the default (half the free device memory at the
 * call). Errors: none. */
int lts_set_adjoint_memory(lts_t* h, uint64_t bytes);

/* Macro steps run as CUDA graphs (default on): the launches of one macro step (Sec. V-B
 * schedule) are captured once per parity of the macro-step index and replayed, with the
 * step's source amplitudes and receiver sample times uploaded before each replay. A graph
 * is re-captured when anything it captured changes (device state, engine, grid shape,
 * buffers); with profiling enabled the launches are issued directly. enable = 0 issues
 * every launch directly. */
int lts_set_graphs(lts_t* h, int enable);

/* Bound of the kernels' asynchronous-completion waits, in SM cycles (default 2e9, about one
 * second): the tensor-core completions and the sparse predict kernel's bulk DOF copies (TMA).
 * suppress_commit != 0 is the failure-path test: the kernels issue no tensor-core work and no
 * copy, so every wait runs out at the bound, the kernel records the timeout, releases its
 * tensor memory and returns; the next synchronising call returns LTS_ERR_TIMEOUT (and clears
 * the report) while the handle stays usable. The DOFs are then undefined. Errors:
 * LTS_ERR_ARG for cycles <= 0. */
int lts_set_wait_limit(lts_t* h, int64_t cycles, int suppress_commit);

/* Autotuner over launch configurations: contraction engine (FP32 CUDA cores, sparse
 * products, split-tf32 tensor cores, and plain tf32 only if allow_tf32) x resident CTAs per
 * SM the predict and neighbour grids are sized for (the occupancy maximum and one fewer) x
 * tile variant (sparse engine: the neighbour kernel's 8 or 4 elements per CTA; other
 * engines: 0). Each candidate advances one macro step from a device-side snapshot of the
 * state, timed with CUDA events on `cuda_stream` after one untimed warm-up step; the state
 * (DOFs, LTS buffers, time, receiver samples) is restored exactly after every trial, so the
 * simulation is unchanged. The fastest candidate becomes the handle's configuration.
 * Outputs (each may be NULL): chosen[4] = (engine, predict CTAs/SM, neighbour CTAs/SM,
 * tile), best_ms, and for the first `cap` candidates table[cap][5] = (engine, CTAs/SM,
 * CTAs/SM, tile, ms); *n_out the number of candidates. Needs device memory for one copy of
 * the state (else LTS_ERR_OOM); synchronises the stream. */
int lts_autotune(lts_t* h, int allow_tf32, void* cuda_stream, int* chosen, double* best_ms, double* table,
                 int cap, int* n_out);

/* Launch shape of the three main kernels, for reports: ctas_per_sm[3] (resident CTAs per
 * SM from the occupancy query; 0 where the kernel does not exist for this shape) and
 * threads[3] (threads per CTA), in the order predict+local (CUDA cores), neighbour,
 * predict+local (tensor cores). Either array may be NULL. */
int lts_launch_config(lts_t* h, int* ctas_per_sm, int* threads);

/* Checkpoint / resume at a macro-step boundary (every cluster has completed its steps and
 * no LTS buffer holds data still to be read, so the DOFs are the whole state). save writes
 * the DOFs of every simulation (FP32 as held on the device), the step counter, the finest
 * step and every receiver's samples so far to `path`; load restores them into a handle
 * set up the same way (mesh, material, sources, receivers, clusters, simulations), so that
 * continuing reproduces the uninterrupted run bitwise. Both synchronise. Errors:
 * LTS_ERR_STATE (no clusters, or not at a macro-step boundary), LTS_ERR_ARG (file not
 * writable / readable, or written for a different set-up). */
int lts_checkpoint_save(lts_t* h, const char* path);
int lts_checkpoint_load(lts_t* h, const char* path);

/* Energy of a caller-owned DOF array, for callers that cannot allocate device memory.
 * The paper has no counterpart: this is an integration aid. Some callers cannot call
 * cudaMalloc once they are running: their device memory belongs to another framework's
 * pool or arena, or they must not risk an allocation failure or the implicit
 * synchronisation of cudaMalloc/cudaFree inside their time loop. This call allocates
 * nothing. Its only scratch is a file-scope device array of LTS_NOALLOC_MAX_ELEMENTS
 * doubles (2 MiB) that every GPU which loads the library holds until the process exits.
 * Inputs (device pointers on the current CUDA device, caller-owned): dofs FP32
 * [n_elem][9 + 6 n_mech][B(order)] (the layout of lts_get_dofs, unpadded), mat FP64
 * [n_elem][4] = (lambda, mu, rho, |det J|). Output: *energy (device FP64) receives
 * sum_k |det J_k| sum_b (rho |v_b|^2/2 + sigma_b : C^-1 sigma_b / 2), the quantity of
 * lts_energy. Runs asynchronously on cuda_stream (NULL = legacy default stream).
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture. The address is
 * kept per device for the life of the process: after a cudaDeviceReset (or any other end of
 * the device's primary context) the kept address is stale, so this entry point must not be
 * called on that device again in the same process. Every call
 * shares the one scratch array, so calls that overlap on the GPU (on different streams)
 * race; the array is fully rewritten for the first n_elem entries by each call, so
 * nothing needs clearing. Errors: LTS_ERR_ARG for a bad order or mechanism count, a NULL
 * pointer, or n_elem <= 0 or n_elem > LTS_NOALLOC_MAX_ELEMENTS; LTS_ERR_CUDA if the
 * address lookup or a launch fails. */
#define LTS_NOALLOC_MAX_ELEMENTS 262144
int lts_energy_noalloc(int order, int n_mech, const float* dofs, const double* mat, int64_t n_elem,
                       double* energy, void* cuda_stream);

/* Host-only helpers (no handle, no GPU). Reference operators of order O in the basis
 * described above (Sec. III-A), from exact polynomial integration:
 *   K[c][i][j]   = int phi_i d(phi_j)/d(xi_c)                     (3 x B x B)
 *   Ft[f][k][m]  = int_{face f} phi_k psi_m                       (4 x B x F)
 *   Fb[j*3+h][k][m] = int psi_m(chi) phi_k(xi_j(chi'(chi, h)))    (12 x B x F)
 * with psi the orthonormal triangle basis (mode (i,j) = [s^i P_i(a)] P_j^(2i+1,0)(b),
 * s = 1-chi2, a = 2chi1/s-1, b = 2chi2-1, ordered by degree then j), the face parameter
 * chi of face f (vertices (A,B,C) of the face table: x = A + chi1 (B-A) + chi2 (C-A)), and
 * for the neighbour matrices the neighbour's face j whose vertex h coincides with the
 * local face's first vertex (vertex m of the local face at neighbour position
 * (h, h+2, h+1)[m] mod 3). Any output may be NULL. Errors: LTS_ERR_ARG. */
int lts_reference_operators(int order, double* K, double* Ft, double* Fb);

/* phi_b(xi_i) for n reference points xi[3n] -> out[n][B]. Errors: LTS_ERR_ARG. */
int lts_eval_basis(int order, int64_t n, const double* xi, double* out);

/* The projection quadrature rule on the reference tetrahedron (collapsed Gauss-Jacobi):
 * *n points, xi[3 *n] and weights w[*n] (either may be NULL to query *n). */
int lts_quadrature_rule(int order, int64_t* n, double* xi, double* w);

#ifdef __cplusplus
}
#endif
#endif /* ADER_LTS_H */
