"""Helpers shared by the GPU parity tests."""
import math

import numpy as np

FP64_RTOL = 1e-9        # FP64 path vs oracle: relative, on distances and forces
FP32_REL_DIAM = 1e-5    # FP32 path vs oracle: absolute error / mesh diameter


def csr_to_dict(rs, j, d, t):
    out = {}
    for i in range(len(rs) - 1):
        for q in range(rs[i], rs[i + 1]):
            out[(i, int(j[q]))] = (float(d[q]), t[q])
    return out


def geodesic_walker(om, face, bary):
    """Landing error of a straightest walk from particle i along tangent t for length d, to
    particle j: a tangent is a valid answer iff it starts a geodesic of that length to j."""
    x = om.world(face, bary)

    def walk(i, j, d, t):
        f2, b2, _, _ = om.shift(int(face[i]), bary[i], d * np.asarray(t), None)
        return float(np.linalg.norm(om.world([f2], [b2])[0] - x[j]))
    return walk


def descent_checker(om, face, bary, r_c):
    """Deficit 1 - (l(i,j) - l(i',j)) / eps where i' is particle i moved by eps along tangent t
    (a straightest walk): 0 for any initial tangent of a shortest path from i to j, also on
    the cut locus and for paths that bend at vertices (first variation of length), and
    1 - cos(angle) for a direction off every such tangent."""
    def check(i, j, d, t):
        eps = 1e-4 * d
        f2, b2, _, _ = om.shift(int(face[i]), bary[i], eps * np.asarray(t), None)
        rc = 2 * d + 1e-12 if not math.isfinite(r_c) else r_c + eps
        d0, _ = om.query(int(face[i]), bary[i], rc, [int(face[j])], [bary[j]])
        d1, _ = om.query(f2, b2, rc, [int(face[j])], [bary[j]])
        return 1.0 - (d0[0] - d1[0]) / eps
    return check


def compare_pairs(gpu, ref, r_c, dist_tol, tan_tol, rel=True, band=None, tie=None, walker=None,
                  land_tol=None):
    """Compare two CSR neighbour sets.  Pairs within `band` of the cutoff may be missing on
    either side.  When ref carries a fifth array (the oracle's tie gap), tangents of pairs
    whose rival geodesic is within `tie` (absolute length) are not compared: at such
    cut-locus points the tangent is set-valued.  Returns (n_compared, max_dist_err,
    max_tan_err).  With `walker`, a tangent that differs from the reference by more than
    tan_tol is still accepted when the walk along it lands within land_tol of the target:
    the pair then lies on the cut locus, where several geodesics of equal length exist."""
    G = csr_to_dict(*gpu)
    R = csr_to_dict(*ref[:4])
    gap = {}
    if len(ref) > 4:
        rs, j, g = ref[0], ref[1], ref[4]
        for i in range(len(rs) - 1):
            for q in range(rs[i], rs[i + 1]):
                gap[(i, int(j[q]))] = float(g[q])
    if band is None:
        band = 1e-9 * r_c if math.isfinite(r_c) else 0.0
    for k in set(G) ^ set(R):
        d = G[k][0] if k in G else R[k][0]
        assert math.isfinite(r_c) and abs(d - r_c) <= band, f"pair {k} only on one side (d={d}, r_c={r_c})"
    md = mt = 0.0
    n = 0
    for k in set(G) & set(R):
        dg, tg = G[k]
        dr, tr = R[k]
        err = abs(dg - dr) / (dr if rel else 1.0)
        md = max(md, err)
        tie_k = tie if tie is not None else (1e-12 * dr)
        if gap.get(k, math.inf) > tie_k:
            e = float(np.linalg.norm(tg - tr))
            if e > tan_tol and walker is not None and walker(k[0], k[1], dg, tg) <= land_tol:
                e = 0.0     # a different, equally valid geodesic
            if e > mt:
                mt, worst = e, (k, dg, dr, gap.get(k, math.inf))
        n += 1
    assert md <= dist_tol, f"distance error {md} > {dist_tol}"
    assert mt <= tan_tol, f"tangent error {mt} > {tan_tol} at pair {worst[0]}: d_gpu={worst[1]!r} " \
                          f"d_ref={worst[2]!r} rival gap={worst[3]!r}"
    return n, md, mt


def select_rows(csr, rows):
    """The CSR rows `rows` (in that order) of a (row_start, j, dist, tangent) result."""
    rs, j, d, t = csr[:4]
    idx = [np.arange(rs[i], rs[i + 1]) for i in rows]
    cnt = np.array([len(a) for a in idx], np.int64)
    out_rs = np.concatenate([[0], np.cumsum(cnt)])
    sel = np.concatenate(idx) if idx else np.zeros(0, np.int64)
    return out_rs, j[sel], d[sel], t[sel]


def sample_sources(n, k, seed):
    """k distinct particle indices (seeded), sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


def force_row_bounds(ref_rows, pot, dudl, delta, tan_err, tie=None):
    """Per-row bound on |F_gpu - F_ref| for forces built from distances within `delta` and
    tangents within `tan_err` of the reference rows (row_start, j, dist, tangent[, gap]):
    each pair moves its U' by at most its variation over [d - delta, d + delta], and turns
    it by tan_err (fully, where the reference reports a rival geodesic within `tie`); pairs
    within delta of the cutoff may be present on one side only."""
    rs, d = ref_rows[0], ref_rows[2]
    gap = ref_rows[4] if len(ref_rows) > 4 else np.full(len(d), np.inf)
    rc = pot["r_cut"]
    edge = abs(dudl(max(rc - delta, 1e-300)))
    out = np.zeros(len(rs) - 1)
    for k in range(len(rs) - 1):
        b = 4.0 * edge
        for q in range(rs[k], rs[k + 1]):
            u = dudl(d[q])
            lo = dudl(d[q] - delta) if d[q] > delta else math.inf
            hi = dudl(d[q] + delta)
            b += max(abs(lo - u), abs(hi - u)) + abs(u) * (2.0 if tie is not None and gap[q] <= tie else tan_err)
        out[k] = b
    return out
