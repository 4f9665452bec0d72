"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed-form values, moment conditions of the delta functions, an independent dense octree
builder, brute-force search, textbook trilinear interpolation (scipy), the discrete adjoint
identity, conservation, finite differences and the convergence order of AB2."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2605_20565_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------
# An independent Morton encoder (magic-number bit spreading, not the oracle's bit loop)
# ---------------------------------------------------------------------------------------

def _spread3(v):
    v = np.asarray(v, np.uint64) & np.uint64(0x1FFFFF)
    for shift, mask in ((32, 0x1F00000000FFFF), (16, 0x1F0000FF0000FF), (8, 0x100F00F00F00F00F),
                        (4, 0x10C30C30C30C30C3), (2, 0x1249249249249249)):
        v = (v | (v << np.uint64(shift))) & np.uint64(mask)
    return v


def morton_np(x, y, z):
    return _spread3(x) | (_spread3(y) << np.uint64(1)) | (_spread3(z) << np.uint64(2))


def test_morton_closed_forms():
    assert oracle.morton(1, 0, 0) == 1
    assert oracle.morton(0, 1, 0) == 2
    assert oracle.morton(0, 0, 1) == 4
    assert oracle.morton(1, 1, 1) == 7
    assert oracle.morton(2, 0, 0) == 8
    assert oracle.morton(3, 3, 3) == 63
    m = (1 << 21) - 1
    assert oracle.morton(m, m, m) == (1 << 63) - 1
    assert oracle.morton(1 << 20, 0, 0) == 1 << 60
    rng = np.random.default_rng(0)
    q = rng.integers(0, 1 << 21, size=(200, 3))
    ref = morton_np(q[:, 0], q[:, 1], q[:, 2])
    for (a, b, c), r in zip(q, ref):
        k = oracle.morton(int(a), int(b), int(c))
        assert k == int(r)
        assert oracle.unmorton(k) == (a, b, c)


# ---------------------------------------------------------------------------------------
# Octree: an independent dense builder on a tiny grid
# ---------------------------------------------------------------------------------------

def _near_surface_np(lo, h, sph):
    """max(0, d_near - r, r - d_far) <= w for boxes [lo, lo+h]^3 (lo: (M, 3))."""
    hi = lo + h
    c = sph[:3]
    e = np.maximum(np.maximum(lo - c, 0.0), c - hi)
    near = np.sqrt(((e[:, 0] ** 2 + e[:, 1] ** 2) + e[:, 2] ** 2))
    f = np.maximum(np.abs(c - lo), np.abs(c - hi))
    far = np.sqrt(((f[:, 0] ** 2 + f[:, 1] ** 2) + f[:, 2] ** 2))
    dist = np.maximum(np.maximum(0.0, near - sph[3]), sph[3] - far)
    return dist <= sph[4]


def dense_build(spheres, lmin, lmax, full=True):
    """Level of the leaf covering each finest cell, on a dense (2^lmax)^3 grid: refine by
    the criterion level by level, then split leaves next to leaves two levels finer until
    none is left; finally list the leaves as (Morton anchor key, level)."""
    n = 1 << lmax
    L = np.full((n, n, n), lmin, np.int64)
    for l in range(lmin, lmax):
        h = 2.0 ** -l
        nl = 1 << l
        idx = np.stack(np.meshgrid(np.arange(nl), np.arange(nl), np.arange(nl), indexing="ij"), -1).reshape(-1, 3)
        blk = 1 << (lmax - l)
        cur = L[idx[:, 0] * blk, idx[:, 1] * blk, idx[:, 2] * blk]
        act = idx[cur == l]
        if act.size == 0:
            continue
        hit = np.zeros(len(act), bool)
        for s in np.asarray(spheres).reshape(-1, 5):
            hit |= _near_surface_np(act * h, h, s)
        for a in act[hit]:
            L[a[0] * blk:(a[0] + 1) * blk, a[1] * blk:(a[1] + 1) * blk, a[2] * blk:(a[2] + 1) * blk] = l + 1
    dirs = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)
            if (dx, dy, dz) != (0, 0, 0) and (full or abs(dx) + abs(dy) + abs(dz) == 1)]
    while True:
        need = np.zeros_like(L)
        for dx, dy, dz in dirs:
            sh = np.full_like(L, -10)
            src = L[max(dx, 0):n + min(dx, 0), max(dy, 0):n + min(dy, 0), max(dz, 0):n + min(dz, 0)]
            sh[max(-dx, 0):n + min(-dx, 0), max(-dy, 0):n + min(-dy, 0), max(-dz, 0):n + min(-dz, 0)] = src
            need = np.maximum(need, sh)
        flag = need >= L + 2
        if not flag.any():
            break
        L0 = L.copy()  # split every flagged leaf of this sweep once
        for c in np.argwhere(flag):
            a = L0[tuple(c)]
            blk = 1 << (lmax - a)
            b0 = (c // blk) * blk
            sl = tuple(slice(b0[d], b0[d] + blk) for d in range(3))
            L[sl] = np.maximum(L[sl], a + 1)
    idx = np.argwhere(np.ones_like(L, bool))
    lev = L.reshape(-1)
    blk = 1 << (lmax - lev)
    anchor = np.all(idx % blk[:, None] == 0, axis=1)
    a = idx[anchor] << (21 - lmax)
    keys = morton_np(a[:, 0], a[:, 1], a[:, 2])
    order = np.argsort(keys)
    return keys[order], lev[anchor][order].astype(np.uint8)


@pytest.mark.parametrize("full", [1, 0])
@pytest.mark.parametrize("case", range(4))
def test_octree_matches_dense_builder(case, full):
    rng = np.random.default_rng(100 + case)
    lmin, lmax = [(1, 5), (2, 5), (2, 4), (1, 4)][case]
    ns = [1, 2, 3, 2][case]
    sph = np.column_stack([rng.uniform(0.2, 0.8, (ns, 3)), rng.uniform(0.05, 0.2, ns), rng.uniform(0.0, 0.08, ns)])
    k, l = oracle.octree_build(sph, lmin, lmax, full)
    kd, ld = dense_build(sph, lmin, lmax, bool(full))
    assert np.array_equal(k, kd)
    assert np.array_equal(l, ld)


def _span(levels):
    return np.uint64(1) << (np.uint64(3) * (np.uint64(21) - levels.astype(np.uint64)))


def check_partition(keys, levels):
    """Leaves tile [0, 8^21) without gaps or overlaps, and every anchor is aligned."""
    sp = _span(levels)
    assert keys[0] == 0
    assert np.all(keys[1:] == keys[:-1] + sp[:-1])
    assert int(keys[-1]) + int(sp[-1]) == 8 ** 21
    assert np.all(keys % sp == 0)


def test_tiny_tree_structure(tiny_tree, tiny_workload):
    k, l = tiny_tree
    w = tiny_workload
    check_partition(k, l)
    assert oracle.count_unbalanced(k, l, 1) == 0
    assert l.min() >= w.lmin and l.max() == w.lmax
    # every coarser leaf fails the refinement criterion (it would otherwise be split)
    cen = oracle.leaf_centres(k, l)
    h = 2.0 ** -l.astype(np.float64)
    lo = cen - 0.5 * h[:, None]
    coarse = l < w.lmax
    for s in w.spheres:
        hits = np.zeros(len(k), bool)
        for lev in np.unique(l[coarse]):
            m = coarse & (l == lev)
            hits[m] = _near_surface_np(lo[m], 2.0 ** -int(lev), s)
        assert not hits.any()
    # the count quoted for this tree (about 5k leaves)
    assert 3000 < k.size < 12000


def test_tree_balance_dense_adjacency(tiny_tree, tiny_workload):
    """Independent 2:1 check: adjacent finest cells never differ by more than one level."""
    k, l = tiny_tree
    lmax = tiny_workload.lmax
    n = 1 << lmax
    L = np.zeros((n, n, n), np.int64)
    cen = oracle.leaf_centres(k, l)
    for c, lev in zip(cen, l):
        b = 1 << (lmax - int(lev))
        i0 = (np.floor(c * n) // b * b).astype(int)
        L[i0[0]:i0[0] + b, i0[1]:i0[1] + b, i0[2]:i0[2] + b] = lev
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                a = L[max(dx, 0):n + min(dx, 0), max(dy, 0):n + min(dy, 0), max(dz, 0):n + min(dz, 0)]
                b = L[max(-dx, 0):n + min(-dx, 0), max(-dy, 0):n + min(-dy, 0), max(-dz, 0):n + min(-dz, 0)]
                assert np.abs(a - b).max() <= 1


def test_count_unbalanced_detects_violation():
    # two leaves of level 1 next to a block refined to level 3: unbalanced by construction
    keys, levels = [], []
    for c in range(8):
        if c == 0:
            for g in range(8):
                for h in range(8):
                    keys.append((g * 8 + h) << (3 * 18))
                    levels.append(3)
        else:
            keys.append(c << (3 * 20))
            levels.append(1)
    k = np.array(keys, np.uint64)
    l = np.array(levels, np.uint8)
    check_partition(k, l)
    assert oracle.count_unbalanced(k, l, 1) > 0


# ---------------------------------------------------------------------------------------
# Host-cell search (Algorithm 1)
# ---------------------------------------------------------------------------------------

def _unmorton_np(keys):
    """Integer anchor coordinates of Morton keys (bit loop in numpy, independent of the oracle)."""
    k = np.asarray(keys, np.uint64)
    out = np.zeros((k.size, 3), np.int64)
    for b in range(21):
        for d in range(3):
            out[:, d] |= ((k >> np.uint64(3 * b + d)) & np.uint64(1)).astype(np.int64) << b
    return out


def paint_host_grid(keys, levels, lmax):
    """Dense (2^lmax)^3 grid holding, in every finest cell, the index of the leaf whose box
    covers it: each leaf paints its own block.  Every cell must be painted exactly once."""
    n = 1 << lmax
    grid = np.full((n, n, n), -1, np.int64)
    cnt = np.zeros((n, n, n), np.int64)
    anc = _unmorton_np(keys) >> (21 - lmax)
    for i, (a, lv) in enumerate(zip(anc, levels)):
        b = 1 << (lmax - int(lv))
        grid[a[0]:a[0] + b, a[1]:a[1] + b, a[2]:a[2] + b] = i
        cnt[a[0]:a[0] + b, a[1]:a[1] + b, a[2]:a[2] + b] += 1
    assert (cnt == 1).all()
    return grid


def test_locate_three_ways(tiny_tree, tiny_workload):
    """The key-order search, the leaf-by-leaf box scan and a lookup in a dense painting of the
    leaves agree on every point (the host is the unique leaf whose half-open box holds it)."""
    k, l = tiny_tree
    w = tiny_workload
    x, y, z = w.particles
    b = oracle.locate_ub(k, l, x, y, z)
    c = oracle.locate_brute(k, l, x, y, z)
    grid = paint_host_grid(k, l, w.lmax)
    cell = np.floor(np.stack([x, y, z]) * (1 << w.lmax)).astype(np.int64)
    a = grid[cell[0], cell[1], cell[2]]
    assert np.array_equal(a, c) and np.array_equal(b, c)
    assert (c >= 0).all()
    # each point inside exactly one leaf: the containing box test counts 1
    cen = oracle.leaf_centres(k, l)
    h = 2.0 ** -l.astype(np.float64)
    lo = cen - 0.5 * h[:, None]
    for p in range(0, x.size, 97):
        pt = np.array([x[p], y[p], z[p]])
        inside = np.all((pt >= lo) & (pt < lo + h[:, None]), axis=1)
        assert inside.sum() == 1 and np.argmax(inside) == c[p]


def test_locate_faces_and_outside(tiny_tree, tiny_workload):
    k, l = tiny_tree
    w = tiny_workload
    cen = oracle.leaf_centres(k, l)
    h = 2.0 ** -l.astype(np.float64)
    lo = cen - 0.5 * h[:, None]  # anchors: points on three faces at once
    x, y, z = lo.T
    for fn in (lambda: oracle.locate_ub(k, l, x, y, z),
               lambda: oracle.locate_brute(k, l, x, y, z)):
        assert np.array_equal(fn(), np.arange(k.size, dtype=np.int32))
    bad = np.array([1.0, -1e-300, np.nan, 2.0, 0.5, 0.5])
    ok = np.array([0.5, 0.5, 0.5, 0.5, np.nextafter(1.0, 0.0), -0.0])
    for fn in (lambda a, b: oracle.locate_ub(k, l, a, b, b),
               lambda a, b: oracle.locate_brute(k, l, a, b, b)):
        r = fn(bad, ok)
        assert list(r[:4]) == [-1, -1, -1, -1]
        assert r[4] >= 0 and r[5] >= 0
    # the last leaf in Morton order holds the point just below (1, 1, 1)
    e = np.array([np.nextafter(1.0, 0.0)])
    assert oracle.locate_ub(k, l, e, e, e)[0] == k.size - 1


# ---------------------------------------------------------------------------------------
# Delta functions (Sec. 2.2)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,kernel", [("peskin4", 2), ("roma3", 3)])
def test_phi_golden_values(name, kernel):
    g = json.load(open(os.path.join(GOLDEN, "delta_kernels.json")))[name]
    r = np.array([v[0] for v in g["values"]])
    ref = np.array([v[1] for v in g["values"]])
    assert np.allclose(oracle.phi(kernel, r), ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("name,kernel,width", [("peskin4", 2, 4), ("roma3", 3, 3)])
def test_phi_moments(name, kernel, width):
    g = json.load(open(os.path.join(GOLDEN, "delta_kernels.json")))[name]
    rng = np.random.default_rng(1)
    s = rng.uniform(-50, 50, 100000)
    if width == 4:
        i0 = np.floor(s) - 1
    else:
        i0 = np.floor(s + 0.5) - 1
    j = i0[:, None] + np.arange(width)[None, :]
    r = s[:, None] - j
    ph = oracle.phi(kernel, r.reshape(-1)).reshape(r.shape)
    assert np.all(ph >= 0)
    assert np.allclose(ph.sum(1), 1.0, atol=1e-14)
    assert np.allclose((r * ph).sum(1), 0.0, atol=1e-13)
    assert np.allclose((ph ** 2).sum(1), g["sum_of_squares"], atol=1e-14)
    if width == 4:  # even and odd sums are 1/2 each (Peskin 2002)
        even = np.where(j % 2 == 0, ph, 0.0).sum(1)
        assert np.allclose(even, 0.5, atol=1e-14)
    # support: zero outside the stencil
    assert np.all(oracle.phi(kernel, np.array([2.0001, -2.5, 3.0, 100.0])) == 0.0)


# ---------------------------------------------------------------------------------------
# IBM interpolation / spreading (Eqs. for u*_k and F(x), Sec. 2.2)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [2, 3])
def test_delta_interp_linear_exact(tiny_tree, tiny_workload, kernel):
    k, l = tiny_tree
    w = tiny_workload
    cen = oracle.leaf_centres(k, l)
    f = synth.linear_field(cen)
    X = w.markers
    u, bad = oracle.interp_delta(k, l, w.lmax, kernel, f, *X)
    assert bad == 0
    ref = synth.linear_field(X.T)[:, :3].T
    assert np.abs(u - ref).max() < 1e-12
    const = np.tile([1.5, -2.0, 0.25, 0.0], (k.size, 1))
    u, _ = oracle.interp_delta(k, l, w.lmax, kernel, const, *X)
    assert np.abs(u - np.array([[1.5], [-2.0], [0.25]])).max() < 1e-13


def test_delta_stencil_outside_finest_is_counted(tiny_tree, tiny_workload):
    k, l = tiny_tree
    w = tiny_workload
    f = np.ones((k.size, 4))
    p = np.array([0.01, 0.99, 0.5])  # a coarse corner region and the domain wall
    _, bad = oracle.interp_delta(k, l, w.lmax, 2, f, p, p, p)
    assert bad > 0


@pytest.mark.parametrize("kernel", [2, 3])
@pytest.mark.parametrize("with_dv", [False, True])
def test_spread_adjoint_and_conservation(tiny_tree, tiny_workload, kernel, with_dv):
    k, l = tiny_tree
    w = tiny_workload
    rng = np.random.default_rng(7)
    X = w.markers
    n = X.shape[1]
    F = rng.normal(size=(3, n))
    h3 = 2.0 ** (-3 * w.lmax)
    dV = rng.uniform(0.5, 2.0, n) * h3 if with_dv else None
    dVv = dV if with_dv else np.full(n, h3)
    f, bad = oracle.spread_delta(k, l, w.lmax, kernel, *X, F, dV)
    assert bad == 0
    # conservation: sum_c f(c) h^3 = sum_k F_k dV_k (only finest cells receive force)
    assert np.allclose((f[:, :3] * h3).sum(0), (F * dVv).sum(1), rtol=1e-12, atol=1e-14)
    assert np.all(f[l < w.lmax] == 0.0)
    # adjoint: <I u, F>_L = <u, S F>_E with weights dV_k and h^3
    uf = np.zeros((k.size, 4))
    uf[:, :3] = rng.normal(size=(k.size, 3))
    Iu, _ = oracle.interp_delta(k, l, w.lmax, kernel, uf, *X)
    lhs = float((Iu * F * dVv).sum())
    rhs = float((uf[:, :3] * f[:, :3]).sum() * h3)
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)) * 10
    # the weights of one marker sum to one
    one = np.zeros((3, n))
    one[0, 0] = 1.0
    f1, _ = oracle.spread_delta(k, l, w.lmax, kernel, *X, one)
    assert abs(f1[:, 0].sum() - 1.0) < 1e-14


# ---------------------------------------------------------------------------------------
# Multi-direct forcing (Sec. 2.2)
# ---------------------------------------------------------------------------------------

def _interp_spread_matrix(k, l, lmax, kernel, X, dV):
    """A = I S on the markers X, column by column from unit marker forces (x component)."""
    nm = X.shape[1]
    A = np.zeros((nm, nm))
    for j in range(nm):
        e = np.zeros((3, nm))
        e[0, j] = 1.0
        f, _ = oracle.spread_delta(k, l, lmax, kernel, *X, e, dV)
        u, _ = oracle.interp_delta(k, l, lmax, kernel, f, *X)
        A[:, j] = u[0]
    return A


@pytest.mark.parametrize("kernel", [2, 3])
def test_mdf_one_round_follows_slip_recursion(tiny_tree, tiny_workload, kernel):
    """One round moves the marker slip s = U - I u to s - A s / rho with A = I S built from
    unit forces: catches a dropped dt or rho, a sign error and a missed correction."""
    k, l = tiny_tree
    w = tiny_workload
    X = np.ascontiguousarray(w.markers[:, :40])
    rng = np.random.default_rng(12)
    u_star = np.zeros((k.size, 4))
    u_star[:, :3] = rng.normal(size=(k.size, 3))
    U = rng.normal(size=(3, X.shape[1]))
    rho, dt = 1.7, 0.3
    h3 = 2.0 ** (-3 * w.lmax)
    dV = rng.uniform(0.5, 2.0, X.shape[1]) * h3
    A = _interp_spread_matrix(k, l, w.lmax, kernel, X, dV)
    u1, f1, slip, bad = oracle.ibm_mdf(k, l, w.lmax, kernel, u_star, X, U, rho, dt, 1, dV=dV)
    assert bad == 0
    I0, _ = oracle.interp_delta(k, l, w.lmax, kernel, u_star, *X)
    I1, _ = oracle.interp_delta(k, l, w.lmax, kernel, u1, *X)
    s0, s1 = U - I0, U - I1
    assert np.abs(s1[0] - (s0[0] - A @ s0[0] / rho)).max() < 1e-12
    assert abs(slip[0] - np.sqrt((s0 ** 2).sum())) < 1e-12 and abs(slip[1] - np.sqrt((s1 ** 2).sum())) < 1e-12
    # the total force of one round is the spread of the marker forces, and it conserves them
    assert np.allclose((f1[:, :3] * h3).sum(0), (s0 / dt * dV).sum(1), rtol=1e-12, atol=1e-14)
    assert np.all(u1[:, 3] == u_star[:, 3])


def test_mdf_slip_decreases_and_fixed_point(tiny_tree, tiny_workload):
    k, l = tiny_tree
    w = tiny_workload
    X = w.markers
    cen = oracle.leaf_centres(k, l)
    u_star = synth.sin_field(cen)
    U = np.zeros((3, X.shape[1]))  # a body at rest
    u, f, slip, bad = oracle.ibm_mdf(k, l, w.lmax, 2, u_star, X, U, 1.0, 1.0, 8)
    assert bad == 0
    assert np.all(np.diff(slip) < 0) and slip[-1] < 0.5 * slip[0]
    # no slip: nothing changes
    Iu, _ = oracle.interp_delta(k, l, w.lmax, 2, u_star, *X)
    u2, f2, slip2, _ = oracle.ibm_mdf(k, l, w.lmax, 2, u_star, X, Iu, 1.0, 1.0, 3)
    assert np.all(f2 == 0.0) and np.array_equal(u2, u_star) and np.all(slip2 == 0.0)


# ---------------------------------------------------------------------------------------
# Periodic box (Sec. 5.2): wrapped stencils and level-mates, mean force
# ---------------------------------------------------------------------------------------

def _uniform_periodic(lev, seed):
    ko, lo = oracle.octree_build(np.zeros((0, 5)), lev, lev)
    nc = 1 << lev
    ii, jj, kk = np.meshgrid(np.arange(nc), np.arange(nc), np.arange(nc), indexing="ij")
    sh = np.uint64(21 - lev)
    keys = morton_np(ii.ravel().astype(np.uint64) << sh, jj.ravel().astype(np.uint64) << sh,
                     kk.ravel().astype(np.uint64) << sh)
    leaf = np.searchsorted(ko, keys).reshape(nc, nc, nc)  # leaf index of cell (i, j, k)
    rng = np.random.default_rng(seed)
    F = rng.normal(size=(nc, nc, nc, 3))
    field = np.zeros((ko.size, 4))
    field[leaf.ravel(), :3] = F.reshape(-1, 3)
    return ko, lo, nc, F, field, rng


@pytest.mark.parametrize("kernel,width", [(2, 4), (3, 3)])
def test_periodic_delta_interp_wraps(kernel, width):
    lev = 4
    ko, lo, nc, F, field, rng = _uniform_periodic(lev, 5)
    P = np.concatenate([rng.uniform(0, 1, (200, 3)), rng.uniform(0, 1.5 / nc, (100, 3)),
                        1.0 - rng.uniform(0, 1.5 / nc, (100, 3))])
    u, bad = oracle.interp_delta(ko, lo, lev, kernel, field, *P.T, periodic=True)
    assert bad == 0
    ref = np.zeros((3, P.shape[0]))
    for p, x in enumerate(P):
        s = x * nc - 0.5
        i0 = (np.floor(s).astype(int) - 1) if kernel == 2 else (np.floor(s + 0.5).astype(int) - 1)
        for a in range(width):
            for b in range(width):
                for c in range(width):
                    w = (oracle.phi(kernel, [s[0] - (i0[0] + a)])[0] * oracle.phi(kernel, [s[1] - (i0[1] + b)])[0] *
                         oracle.phi(kernel, [s[2] - (i0[2] + c)])[0])
                    ref[:, p] += w * F[(i0[0] + a) % nc, (i0[1] + b) % nc, (i0[2] + c) % nc]
    assert np.abs(u - ref).max() < 1e-12
    # non-periodic: the same points near the walls lose stencil cells
    _, bad_np = oracle.interp_delta(ko, lo, lev, kernel, field, *P.T)
    assert bad_np > 0


def test_periodic_trilinear_matches_wrapped_grid():
    from scipy.interpolate import RegularGridInterpolator
    lev = 4
    ko, lo, nc, F, field, rng = _uniform_periodic(lev, 6)
    Fp = np.pad(F, ((1, 1), (1, 1), (1, 1), (0, 0)), mode="wrap")
    g = (np.arange(-1, nc + 1) + 0.5) / nc
    P = np.concatenate([rng.uniform(0, 1, (300, 3)), rng.uniform(0, 0.5 / nc, (100, 3)),
                        1.0 - rng.uniform(1e-9, 0.5 / nc, (100, 3))])
    host = oracle.locate_ub(ko, lo, *P.T)
    u = oracle.interp_trilinear(ko, lo, field, *P.T, host, periodic=True)
    ref = np.stack([RegularGridInterpolator((g, g, g), Fp[..., d])(P) for d in range(3)])
    assert np.abs(u - ref).max() < 1e-12


def test_periodic_spread_conserves_at_walls():
    lev = 4
    ko, lo, nc, F, field, rng = _uniform_periodic(lev, 7)
    X = np.concatenate([rng.uniform(0, 1.0 / nc, (50, 3)), 1.0 - rng.uniform(1e-9, 1.0 / nc, (50, 3))]).T
    Fk = rng.normal(size=(3, X.shape[1]))
    f, bad = oracle.spread_delta(ko, lo, lev, 2, *X, Fk, periodic=True)
    assert bad == 0
    h3 = 2.0 ** (-3 * lev)
    assert np.allclose((f[:, :3] * h3).sum(0), (Fk * h3).sum(1), rtol=1e-12, atol=1e-14)
    # adjoint with wrapping
    Iu, _ = oracle.interp_delta(ko, lo, lev, 2, field, *X, periodic=True)
    assert abs((Iu * Fk).sum() - (field[:, :3] * f[:, :3]).sum()) < 1e-10 * max(1.0, abs((Iu * Fk).sum()))


def test_field_mean(tiny_tree):
    k, l = tiny_tree
    rng = np.random.default_rng(4)
    c = np.tile([0.5, -2.0, 3.0, 0.0], (k.size, 1))
    assert np.allclose(oracle.field_mean(l, c), [0.5, -2.0, 3.0], rtol=1e-13)
    f = rng.normal(size=(k.size, 4))
    vol = 2.0 ** (-3 * l.astype(np.float64))
    assert np.allclose(oracle.field_mean(l, f), (f[:, :3] * vol[:, None]).sum(0), rtol=1e-12)


# ---------------------------------------------------------------------------------------
# Rigid bodies: internal-marker momenta and IBM force / torque sums (Sec. 2.3)
# ---------------------------------------------------------------------------------------

def test_body_sums_closed_forms():
    rng = np.random.default_rng(3)
    cs = np.array([[0.3, 0.4, 0.5], [0.7, 0.6, 0.35]])
    ds = np.array([0.1, 0.06])
    h = 1.0 / 256
    X, start = synth.internal_markers(cs, ds, h)
    w = h ** 3
    rho = 1.3
    xb = cs
    body = np.repeat(np.arange(2), np.diff(start))
    r = X - cs[body].T
    # uniform translation: P = rho V U, and no angular momentum (the lattice is symmetric)
    U0 = np.array([0.2, -0.1, 0.35])
    v = np.tile(U0[:, None], (1, X.shape[1]))
    lin, ang = oracle.body_sums(X, v, start, xb, rho, w=w)
    for b in range(2):
        nb = start[b + 1] - start[b]
        assert np.allclose(lin[b], rho * nb * w * U0, rtol=1e-12)
        assert np.abs(ang[b]).max() < 1e-12 * nb * w
    # rigid rotation u = Omega x r: L = rho I Omega with I = sum w (|r|^2 1 - r r^T) (tensor form)
    Om = rng.normal(size=3)
    v = np.cross(Om[:, None], r, axis=0)
    lin, ang = oracle.body_sums(X, v, start, xb, rho, dV=np.full(X.shape[1], w))
    for b in range(2):
        rb = r[:, start[b]:start[b + 1]]
        I = w * ((rb ** 2).sum() * np.eye(3) - rb @ rb.T)
        assert np.allclose(ang[b], rho * I @ Om, rtol=1e-10)
        assert np.abs(lin[b]).max() < 1e-12
    # IBM force through the centre (F parallel to r): no torque; total force summed with sign
    F = r * rng.uniform(0.5, 2.0, X.shape[1])
    lin, ang = oracle.body_sums(X, F, start, xb, -1.0, w=w)
    assert np.abs(ang).max() < 1e-14
    assert np.allclose(lin[0], -w * F[:, :start[1]].sum(1), rtol=1e-12, atol=1e-16)


# ---------------------------------------------------------------------------------------
# Trilinear interpolation of point particles (Sec. 2.3.2)
# ---------------------------------------------------------------------------------------

def test_trilinear_uniform_tree_matches_scipy():
    from scipy.interpolate import RegularGridInterpolator
    lev = 4
    k, l = oracle.octree_build(np.zeros((0, 5)), lev, lev)
    n = 1 << lev
    cen = oracle.leaf_centres(k, l)
    rng = np.random.default_rng(3)
    vals = rng.normal(size=(k.size, 4))
    vals[:, 3] = 0
    grid = np.zeros((n, n, n, 3))
    ij = np.floor(cen * n).astype(int)
    grid[ij[:, 0], ij[:, 1], ij[:, 2]] = vals[:, :3]
    ax = (np.arange(n) + 0.5) / n
    P = rng.uniform(0, 1, (5000, 3))
    P[:10] = [[0.001, 0.5, 0.999], [0.999, 0.999, 0.999], [0, 0, 0], [0.5, 0.5, 0.5],
              [1 / 32, 1 / 32, 1 / 32], [0.25, 0.75, 0.5], [0.2, 0.0, 0.9], [0.96, 0.03, 0.5],
              [0.5 + 1 / 32, 0.5, 0.5], [0.3, 0.3, 0.3]]
    host = oracle.locate_ub(k, l, *P.T)
    u = oracle.interp_trilinear(k, l, vals, *P.T, host)
    Pc = np.clip(P, ax[0], ax[-1])  # constant extrapolation in the boundary half-cells
    for d in range(3):
        ref = RegularGridInterpolator((ax, ax, ax), grid[..., d])(Pc)
        assert np.abs(u[d] - ref).max() < 1e-13


def _levelmate_kinds(k, l, P, host):
    """For each point: True when every level-mate is in the domain and not covered by a
    coarser leaf (found by brute force on the leaf boxes)."""
    cen = oracle.leaf_centres(k, l)
    hl = l[host].astype(int)
    ok = np.ones(len(P), bool)
    h = 2.0 ** -hl
    c = np.floor(P * (2.0 ** hl)[:, None])
    t = P * (2.0 ** hl)[:, None] - (c + 0.5)
    s = np.where(t >= 0, 1, -1)
    for corner in range(8):
        off = np.array([(corner >> d) & 1 for d in range(3)])
        m = c + off * s
        inside = np.all((m >= 0) & (m < (2.0 ** hl)[:, None]), axis=1)
        ok &= inside
        mc = (m + 0.5) * h[:, None]
        mc = np.clip(mc, 0, np.nextafter(1, 0))
        leaf = oracle.locate_brute(k, l, *mc.T)
        ok &= l[leaf] >= hl
    return ok


def test_trilinear_linear_exact_and_constant(tiny_tree, tiny_workload):
    k, l = tiny_tree
    w = tiny_workload
    P = w.particles.T[:4000]
    host = oracle.locate_ub(k, l, *P.T)
    cen = oracle.leaf_centres(k, l)
    u = oracle.interp_trilinear(k, l, synth.linear_field(cen), *P.T, host)
    ref = synth.linear_field(P)[:, :3].T
    ok = _levelmate_kinds(k, l, P, host)
    assert ok.sum() > 1000
    # refined level-mates included: their volume-weighted means are centre values of a
    # linear field, so exactness holds wherever no level-mate is hanging or outside
    assert np.abs(u[:, ok] - ref[:, ok]).max() < 1e-12
    const = np.tile([0.5, 1.0, -3.0, 0.0], (k.size, 1))
    u = oracle.interp_trilinear(k, l, const, *P.T, host)
    assert np.abs(u - np.array([[0.5], [1.0], [-3.0]])).max() < 1e-13


def test_trilinear_refined_levelmate_case_is_exercised(tiny_tree, tiny_workload):
    """Points in level-4 leaves next to level-5 leaves: some level-mates are refined and
    the linear-exactness pin covers them."""
    k, l = tiny_tree
    w = tiny_workload
    P = w.particles.T
    host = oracle.locate_ub(k, l, *P.T)
    hl = l[host].astype(int)
    c = np.floor(P * (2.0 ** hl)[:, None])
    t = P * (2.0 ** hl)[:, None] - (c + 0.5)
    s = np.where(t >= 0, 1, -1)
    n_ref = 0
    for corner in range(1, 8):
        off = np.array([(corner >> d) & 1 for d in range(3)])
        m = c + off * s
        inside = np.all((m >= 0) & (m < (2.0 ** hl)[:, None]), axis=1)
        mc = np.clip((m + 0.5) * (2.0 ** -hl)[:, None], 0, np.nextafter(1, 0))
        leaf = oracle.locate_brute(k, l, *mc.T)
        n_ref += int((inside & (l[leaf] > hl)).sum())
    assert n_ref > 100


def test_trilinear_hanging_takes_coarse_value():
    """Reading check (parity unpinned by the paper): with a field that is 1 on one coarse
    leaf and 0 elsewhere, a fine point next to it receives exactly the weights of the
    level-mates that fall inside that leaf."""
    # level-1 tree with octant 0 refined to level 2
    keys = [(g << (3 * 19)) for g in range(8)] + [(c << (3 * 20)) for c in range(1, 8)]
    levels = [2] * 8 + [1] * 7
    k = np.array(keys, np.uint64)
    l = np.array(levels, np.uint8)
    f = np.zeros((k.size, 4))
    f[8 + 0, 0] = 1.0  # octant 1 (x high): the level-1 leaf at key 1<<60
    P = np.array([[0.45, 0.1, 0.1]])  # in the level-2 leaf (1,0,0); x-mate is (2,0,0): in octant 1
    host = oracle.locate_ub(k, l, *P.T)
    assert l[host[0]] == 2
    u = oracle.interp_trilinear(k, l, f, *P.T, host)
    tx = 0.45 * 4 - 1.5  # t_x = 0.3 -> weight of the x-mate is 0.3
    assert abs(u[0, 0] - abs(tx)) < 1e-14


# ---------------------------------------------------------------------------------------
# Learned-index root network gradient
# ---------------------------------------------------------------------------------------

def test_mlp_gradient_central_differences():
    rng = np.random.default_rng(11)
    prm = rng.normal(scale=0.5, size=oracle.MLP_NPARAM)
    x = rng.uniform(0, 1, 64)
    t = np.sort(rng.uniform(0, 1, 64))
    loss, g = oracle.mlp_loss_grad(prm, x, t)
    y = oracle.mlp_forward(prm, x)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-14
    eps = 1e-6
    num = np.empty_like(g)
    for i in range(prm.size):
        a, b = prm.copy(), prm.copy()
        a[i] += eps
        b[i] -= eps
        num[i] = (oracle.mlp_loss_grad(a, x, t)[0] - oracle.mlp_loss_grad(b, x, t)[0]) / (2 * eps)
    assert np.allclose(g, num, rtol=1e-6, atol=1e-8)


# ---------------------------------------------------------------------------------------
# AB2 advection (Sec. 2.3.2)
# ---------------------------------------------------------------------------------------

def _relax(dt, steps, tau=0.5):
    st = {"x": np.zeros((3, 1)), "v": np.zeros((3, 1)), "a_prev": np.zeros((3, 1)), "v_prev": np.zeros((3, 1))}
    u = np.array([[1.0], [0.0], [-2.0]])
    for s in range(steps):
        oracle.advect_ab2(st, u, tau, 0.0, dt, s == 0)
    t = dt * steps
    vex = u[:, 0] * (1 - math.exp(-t / tau))
    xex = u[:, 0] * (t - tau * (1 - math.exp(-t / tau)))
    return np.abs(st["v"][:, 0] - vex).max(), np.abs(st["x"][:, 0] - xex).max()


def test_ab2_second_order_relaxation():
    e1 = _relax(0.01, 100)
    e2 = _relax(0.005, 200)
    e3 = _relax(0.0025, 400)
    for i in range(2):
        r1, r2 = e1[i] / e2[i], e2[i] / e3[i]
        assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0  # error ratio about 4: second order
    assert e3[0] < 1e-4


def test_ab2_uniform_motion_exact():
    st = {"x": np.full((3, 2), 0.25), "v": np.array([[0.1, -0.2]] * 3), "a_prev": np.zeros((3, 2)),
          "v_prev": np.zeros((3, 2))}
    u = st["v"].copy()  # fluid moves with the particle: no drag
    for s in range(10):
        oracle.advect_ab2(st, u, 1.0, 0.0, 0.01, s == 0)
    assert np.allclose(st["x"], 0.25 + 0.1 * np.array([[1, -2]] * 3) * 0.1 * 1, atol=1e-15)


def test_ab2_schiller_naumann_factor():
    st = {"x": np.zeros((3, 1)), "v": np.zeros((3, 1)), "a_prev": np.zeros((3, 1)), "v_prev": np.zeros((3, 1))}
    u = np.array([[2.0], [0.0], [0.0]])
    oracle.advect_ab2(st, u, 1.0, 3.0, 0.1, True)
    fp = 1 + 0.15 * (3.0 * 2.0) ** 0.687
    assert abs(st["v"][0, 0] - 0.1 * fp * 2.0) < 1e-14


def _state(x, v):
    x = np.array(x, np.float64).reshape(3, -1).copy()
    v = np.array(v, np.float64).reshape(3, -1).copy()
    return {"x": x, "v": v, "a_prev": np.zeros_like(x), "v_prev": np.zeros_like(x)}


def test_ab2_periodic_crossings_exact():
    """Periodic box (Sec. 5.2): a particle leaving through one face re-enters through the
    opposite one.  Values chosen so that every sum is exact in binary: an Euler step with the
    fluid moving with the particle (no drag) moves x by dt v exactly."""
    # per column: start, velocity, wrapped result (dt = 1)
    cases = [(0.75, 0.5, 0.25),          # crosses x = 1 upwards
             (0.25, -0.5, 0.75),         # crosses x = 0 downwards
             (0.5, 0.5, 0.0),            # lands exactly on x = 1: the image is 0
             (0.0, -0.25, 0.75),         # leaves from the face x = 0
             (1.0 - 2.0 ** -10, 2.0 ** -9, 2.0 ** -10),
             (0.375, 0.125, 0.5)]        # stays inside: untouched
    x0 = np.array([c[0] for c in cases])
    v0 = np.array([c[1] for c in cases])
    ref = np.array([c[2] for c in cases])
    for axis in range(3):
        x = np.full((3, len(cases)), 0.5)
        v = np.zeros((3, len(cases)))
        x[axis], v[axis] = x0, v0
        st = _state(x, v)
        oracle.advect_ab2(st, st["v"].copy(), 1.0, 0.0, 1.0, True, periodic=True)
        assert np.array_equal(st["x"][axis], ref)
        others = [d for d in range(3) if d != axis]
        assert np.array_equal(st["x"][others], np.full((2, len(cases)), 0.5))
        assert np.array_equal(st["v"], v)  # the wrap moves positions only


def test_ab2_periodic_rounds_to_zero_not_one():
    """x just below 0 by less than half an ulp of 1 has the image 1 - 2^-60, which rounds to
    1.0 in FP64; the wrapped position must still lie in [0, 1): it becomes 0."""
    st = _state([[0.0], [0.5], [0.5]], [[-2.0 ** -60], [0.0], [0.0]])
    oracle.advect_ab2(st, st["v"].copy(), 1.0, 0.0, 1.0, True, periodic=True)
    assert st["x"][0, 0] == 0.0


def test_ab2_periodic_differs_from_free_by_whole_turns():
    """On random states with drag, the periodic step gives the free step's positions shifted by
    whole turns into [0, 1), and identical velocities and histories."""
    rng = np.random.default_rng(7)
    n = 4000
    x = rng.uniform(0.0, 1.0, (3, n))
    v = rng.normal(0.0, 0.3, (3, n))
    u = rng.normal(0.0, 0.3, (3, n))
    free, per = _state(x, v), _state(x, v)
    for s in range(3):
        oracle.advect_ab2(free, u, 0.7, 2.0, 0.05, s == 0)
        oracle.advect_ab2(per, u, 0.7, 2.0, 0.05, s == 0, periodic=True)
        # the periodic run restarts from its own (wrapped) positions: compare one step at a time
        for key in ("v", "a_prev", "v_prev"):
            assert np.array_equal(free[key], per[key])
        assert ((per["x"] >= 0.0) & (per["x"] < 1.0)).all()
        turns = free["x"] - per["x"]
        assert np.allclose(turns, np.round(turns), rtol=0, atol=4e-16)
        crossed = np.round(turns) != 0
        assert crossed.any()
        free["x"] = per["x"].copy()
