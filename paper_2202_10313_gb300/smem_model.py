"""Shared-memory wavefront model of the forward kernels' main loops (analysis tool, no GPU).

An SM's shared memory serves one wavefront per cycle. The model counts, per warp instruction
of the main loops, the wavefronts a load needs: a 16-byte load is served in four phases of 8
threads, an 8-byte load in two phases of 16, a 4-byte load in one phase of 32; within a phase
identical addresses broadcast and distinct 16/8/4-byte chunks cost one wavefront per chunk
that falls into the same bank group (8 groups of 4 banks for 16-byte chunks, 16 pairs for
8-byte, 32 banks for 4-byte). Threads follow the kernels' task orders (mode columns by
degree, highest first; face-mode pairs with the pair index slowest), each thread walking its
own k- or face-mode range in step with the others of its warp.

Covered: the time-kernel products (per derivative), the volume product, the local-surface
product and the F^ projection of k_predict_local, and the neighbour product of k_neighbour.
Not covered: staging stores, the split partial exchange, per-element coefficient loads.

    python -m paper_2202_10313_gb300.smem_model [--order 5]
"""
import argparse


def nbasis(o):
    return o * (o + 1) * (o + 2) // 6


def nface(o):
    return o * (o + 1) // 2


def face_degree(f):
    q = 0
    while nface(q + 1) <= f:
        q += 1
    return q


def wavefronts(lane_addrs, width):
    """Wavefronts of one warp load: lane_addrs = [(lane, float address)], width in floats."""
    per_phase = 32 // width if width > 1 else 32
    groups = 32 // width
    total = 0
    for ph in range(0, 32, per_phase):
        chunks = {a // width for (l, a) in lane_addrs if ph <= l < ph + per_phase}
        if not chunks:
            continue
        count = {}
        for c in chunks:
            count[c % groups] = count.get(c % groups, 0) + 1
        total += max(count.values())
    return total


def run(threads):
    """threads: per thread a list of iterations, each a list of (float address, width) loads
    (the same load sequence for every thread). Sums the wavefronts warp by warp, iteration by
    iteration, over the threads still inside their range."""
    total = 0
    for w in range(0, len(threads), 32):
        warp = threads[w:w + 32]
        n = max((len(t) for t in warp), default=0)
        for it in range(n):
            active = [(lane, t[it]) for lane, t in enumerate(warp) if it < len(t)]
            if not active:
                continue
            for j in range(len(active[0][1])):
                total += wavefronts([(lane, loads[j][0]) for lane, loads in active], active[0][1][j][1])
    return total


def column_tasks(order, ne, nt):
    """(slot, mode column, degree) per thread, columns by degree, highest first."""
    out = []
    for q in range(order - 1, -1, -1):
        np_ = (q + 1) * (q + 2) // 2
        for idx in range(ne * np_):
            out.append((idx // np_, nbasis(q) + idx % np_, q))
    out += [None] * (nt - len(out))
    return out


def predict_model(order=5, elastic=False, k_layout="planes", surface="pairs", ne=7, ar=12, fr=12):
    """Wavefronts per element of k_predict_local's main loops. k_layout: 'planes' (three K_c
    planes, 4-byte loads) or 'interleaved' (one 16-byte load of the three K_c entries);
    surface: 'pairs' (two face modes per thread, pair index slowest) or 'single' (one face
    mode per thread, modes by degree, highest first, the mode fastest within a face)."""
    B, F = nbasis(order), nface(order)
    nt = -(-ne * B // 32) * 32
    bs = B if B % 2 else B + 1
    ks = bs + 2
    nsplit = nbasis(order - 2)
    fls = 4 * F * fr
    tasks = column_tasks(order, ne, nt)

    def k_loads(col, k, transposed):
        r, c = (k, col) if transposed else (col, k)
        if k_layout == "planes":
            return [((cc * B + r) * ks + c, 1) for cc in range(3)]
        return [((r * bs + c) * 4, 4)]

    def x_loads(e, k):
        base = e * B * ar + k * ar
        return [(base, 4), (base + 4, 4), (base + 8, 1)]

    def kmid(kb, kend):
        return max(kb, (kb + kend + 1) // 2)

    time_total = 0
    for d in range(order - 1):
        kend = nbasis(order - d) if elastic else B
        threads = []
        for t in tasks:
            if t is None:
                threads.append([])
                continue
            e, b, p = t
            hj = b - nbasis(order - 1)
            if p == order - 1 and hj < nsplit:
                ph = 0
                while nbasis(ph + 1) <= hj:
                    ph += 1
                col, k0, k1 = hj, kmid(nbasis(ph + 1), kend), kend
            elif b < nsplit:
                col, k0, k1 = b, nbasis(p + 1), kmid(nbasis(p + 1), kend)
            else:
                col, k0, k1 = b, nbasis(p + 1), kend
            threads.append([x_loads(e, k) + k_loads(col, k, False) for k in range(k0, k1)])
        time_total += run(threads)
    vol = run([[] if t is None else [x_loads(t[0], k) + k_loads(t[1], k, True) for k in range(nbasis(t[2]))]
               for t in tasks])
    surf = 0
    if surface == "pairs":
        # face-mode pairs (F-1-2a, F-2-2a), pair index slowest, then slot, then face
        npair = (F + 1) // 2
        pair_tasks = [(e, i, a) for a in range(npair) for e in range(ne) for i in range(4)]
        for p0 in range(0, len(pair_tasks), nt):
            threads = []
            for e, i, a in pair_tasks[p0:p0 + nt]:
                f1 = F - 1 - 2 * a
                f2 = f1 - 1 if f1 >= 1 else f1
                threads.append([x_loads(e, k) + [(i * B * F + k * F + f1, 1), (i * B * F + k * F + f2, 1)]
                                for k in range(nbasis(face_degree(f2)), B)])
            surf += run(threads)
    else:
        single = []
        for q in range(order - 1, -1, -1):
            for idx in range(ne * 4 * (q + 1)):
                r = idx % (4 * (q + 1))
                single.append((idx // (4 * (q + 1)), r // (q + 1), nface(q) + r % (q + 1), q))
        for p0 in range(0, len(single), nt):
            surf += run([[x_loads(e, k) + [(i * B * F + k * F + f, 1)] for k in range(nbasis(q), B)]
                         for e, i, f, q in single[p0:p0 + nt]])
    proj = run([[] if t is None else
                [[(t[0] * fls + (i * F + f) * fr, 4), (t[0] * fls + (i * F + f) * fr + 4, 2),
                  ((i * F + f) * B + t[1], 1)] for i in range(4) for f in range(nface(t[2] + 1))]
                for t in tasks])
    per = lambda x: x / ne
    return {"time": per(time_total), "volume": per(vol), "local_surface": per(surf), "projection": per(proj),
            "total": per(time_total + vol + surf + proj)}


def neighbour_product_model(order=5, ne=8, xr=10, jh=None):
    """Wavefronts per element of k_neighbour's F- product (face-mode pairs, pair index slowest);
    jh[e][i]: the (j, h) table each face uses (a fixed pattern by default)."""
    B, F = nbasis(order), nface(order)
    nt = -(-ne * B // 32) * 32
    npair = (F + 1) // 2
    jh = jh or [[(3 * e + 5 * i) % 12 for i in range(4)] for e in range(ne)]
    tasks = [(e, i, a) for a in range(npair) for e in range(ne) for i in range(4)]
    total = 0
    for p0 in range(0, len(tasks), nt):
        threads = []
        for e, i, a in tasks[p0:p0 + nt]:
            f1 = F - 1 - 2 * a
            f2 = f1 - 1 if f1 >= 1 else f1
            xb, fb = (e * 4 + i) * B * xr, jh[e][i] * B * F
            its = []
            for k in range(nbasis(face_degree(f2)), B):
                x = xb + k * xr
                rows = ([(x, 2), (x + 2, 2), (x + 4, 2), (x + 6, 2), (x + 8, 1)] if xr % 2 == 0
                        else [(x + r, 1) for r in range(9)])
                its.append(rows + [(fb + k * F + f1, 1), (fb + k * F + f2, 1)])
            threads.append(its)
        total += run(threads)
    return total / ne


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--order", type=int, default=5)
    a = ap.parse_args()
    for layout, surface in (("interleaved", "single"), ("interleaved", "pairs"), ("planes", "pairs")):
        m = predict_model(a.order, k_layout=layout, surface=surface)
        print("k_predict_local, K_c %s, surface %s: " % (layout, surface)
              + ", ".join("%s %.0f" % kv for kv in m.items()), "wavefronts per element")
    print("k_neighbour F- product: %.0f wavefronts per element" % neighbour_product_model(a.order))


if __name__ == "__main__":
    main()
