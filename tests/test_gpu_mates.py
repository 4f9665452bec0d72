"""The level-mate table (trilinear level-mates resolved once per octree) on the GPU: every
trilinear result with the table equals the per-query search bit for bit -- single op (FP32 and
FP64, given hosts or searched, plain and learned) and batched (every launch shape, ordered
points) -- and matches the FP64 oracle within the FP32 tolerance, on trees whose refined
level-mates fall in the dense pyramid and below it, on a uniform tree, on random 2:1 trees, and
in the periodic cube (the table is rebuilt when the setting changes)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


@pytest.fixture(scope="module")
def ot():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_20565_gb300 as m
    return m


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def pts(a):
    return [dev(np.ascontiguousarray(a[d], dtype=np.float64)) for d in range(3)]


def rel_err(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def face_points(ko, lo, rng, n):
    """Points on leaf faces, edges and corners (the level-mate octant flips there), at leaf
    centres, near the cube's faces, and uniform."""
    idx = rng.integers(0, ko.size, n)
    h = 2.0 ** -lo[idx].astype(np.float64)
    cen = oracle.leaf_centres(ko, lo)[idx]
    corner = cen + h[:, None] * rng.choice([-0.5, 0.0, 0.5], size=(n, 3))
    near = np.concatenate([rng.uniform(0, 1e-3, (n // 4, 3)), 1.0 - rng.uniform(1e-12, 1e-3, (n // 4, 3))])
    P = np.concatenate([corner, cen, near, rng.uniform(0, 1, (n, 3))])
    return P[np.all((P >= 0) & (P < 1), axis=1)]


@pytest.fixture(scope="module")
def deep(ot):
    sph = np.array([[0.53, 0.47, 0.51, 0.05, 0.02], [0.2, 0.7, 0.3, 0.03, 0.015]])
    ko, lo = oracle.octree_build(sph, 3, 9)
    rng = np.random.default_rng(191)
    d = rng.normal(size=(20000, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    which = rng.integers(0, 2, 20000)
    rad = sph[which, 3] + rng.uniform(-3, 3, 20000) * sph[which, 4]
    P = np.concatenate([sph[which, :3] + d * rad[:, None], face_points(ko, lo, rng, 6000)])
    P = P[np.all((P >= 0) & (P < 1), axis=1)]
    from paper_2605_20565_gb300 import synth
    field = synth.sin_field(oracle.leaf_centres(ko, lo))
    return sph, ko, lo, P, field


def both(ot, tree, fn):
    """fn() without and with the table (the table is freed again afterwards)."""
    ot.ot_octree_build_mates(tree, False)
    a = fn()
    ot.ot_octree_build_mates(tree, True)
    assert ot.ot_octree_has_mates(tree)
    b = fn()
    ot.ot_octree_build_mates(tree, False)
    assert not ot.ot_octree_has_mates(tree)
    return a, b


@pytest.mark.parametrize("map_level", [-1, 0, 8])
def test_single_op_bit_identical_and_oracle(ot, deep, map_level):
    import torch
    sph, ko, lo, P, field = deep
    t = ot.ot_octree_build(sph, 3, 9)
    if map_level >= 0:
        ot.ot_octree_set_map_level(t, map_level)
    href = oracle.locate_ub(ko, lo, *P.T)
    f32 = field.astype(np.float32)
    x, y, z = pts(P.T)

    def run():
        h = torch.empty(P.shape[0], dtype=torch.int32, device="cuda")
        u = ot.ot_interpolate(t, ot.OT_TRILINEAR, x, y, z, dev(f32), host_out=h)
        u2 = ot.ot_interpolate(t, ot.OT_TRILINEAR, x, y, z, dev(f32), host_in=h)
        u64 = ot.ot_interpolate_f64(t, ot.OT_TRILINEAR, x, y, z, dev(field))
        return u, h, u2, u64

    (u, h, u2, u64), (um, hm, u2m, u64m) = both(ot, t, run)
    assert torch.equal(u, um) and torch.equal(h, hm) and torch.equal(u2, u2m) and torch.equal(u64, u64m)
    assert torch.equal(um, u2m)
    assert np.array_equal(hm.cpu().numpy(), href)
    ref32 = oracle.interp_trilinear(ko, lo, f32.astype(np.float64), *P.T, href)
    assert rel_err(um.cpu().numpy(), ref32) <= TOL32
    assert rel_err(u64m.cpu().numpy(), oracle.interp_trilinear(ko, lo, field, *P.T, href)) <= TOL64
    assert ot.ot_last_error(t) & ot.OT_DEV_OUTSIDE == 0


def test_learned_search_with_table(ot, deep):
    import torch
    sph, ko, lo, P, field = deep
    t = ot.ot_octree_build(sph, 3, 9)
    ot.ot_index_train(t, root=ot.OT_ROOT_MLP, n_leaf_models=4096, n_mid_models=64, epochs=1, batch=16384)
    f32 = dev(field.astype(np.float32))
    x, y, z = pts(P.T)

    def run():
        h = torch.empty(P.shape[0], dtype=torch.int32, device="cuda")
        return ot.ot_interpolate(t, ot.OT_TRILINEAR, x, y, z, f32, search=ot.OT_LEARNED, host_out=h), h

    (u, h), (um, hm) = both(ot, t, run)
    assert torch.equal(u, um) and torch.equal(h, hm)
    assert np.array_equal(hm.cpu().numpy(), oracle.locate_ub(ko, lo, *P.T))


@pytest.mark.parametrize("search", [0, 1])
def test_batch_bit_identical_every_shape(ot, deep, search):
    """Every launch shape of the batch (both register budgets, ordered points) with and without
    the table, markers and particles together."""
    import torch
    sph, ko, lo, P, field = deep
    t = ot.ot_octree_build(sph, 3, 9)
    if search == 1:
        ot.ot_index_train(t, root=ot.OT_ROOT_MLP, n_leaf_models=4096, epochs=1, batch=16384)
    f32 = dev(field.astype(np.float32))
    x, y, z = pts(P.T)
    rng = np.random.default_rng(5)
    c = sph[0, :3]
    dirs = rng.normal(size=(3, 2000))
    M = c[:, None] + sph[0, 3] * dirs / np.linalg.norm(dirs, axis=0)
    mx, my, mz = pts(M)
    shapes = [dict(), dict(blocks_per_sm=2), dict(block=128, tile=1), dict(order_level=8, tile=8),
              dict(tri_tile=1, tri_blocks_per_sm=1), dict(tile=2, tri_tile=8, tri_blocks_per_sm=4),
              dict(tri_records=-1), dict(tri_records=-1, order_level=8)]

    def run():
        outs = []
        for lp in shapes:
            up = torch.full((3, P.shape[0]), 7.0, device="cuda")
            hp = torch.full((P.shape[0],), -5, dtype=torch.int32, device="cuda")
            um = torch.full((3, M.shape[1]), 7.0, device="cuda")
            b = ot.ot_batch_create(t, [dict(kernel=ot.OT_PESKIN4, x=mx, y=my, z=mz, u=um),
                                       dict(kernel=ot.OT_TRILINEAR, x=x, y=y, z=z, u=up, host=hp)], f32,
                                   search=search, launch=lp)
            ot.ot_batch_run(b)
            ot.ot_batch_run(b)
            torch.cuda.synchronize()
            ot.ot_batch_destroy(b)
            outs.append((up, hp, um))
        return outs

    plain, mates = both(ot, t, run)
    for (a, ha, ma), (b, hb, mb) in zip(plain, mates):
        assert torch.equal(a, b) and torch.equal(ha, hb) and torch.equal(ma, mb)
    ref = ot.ot_interpolate(t, ot.OT_TRILINEAR, x, y, z, f32)
    assert torch.equal(mates[0][0], ref)
    assert np.array_equal(mates[0][1].cpu().numpy(), oracle.locate_ub(ko, lo, *P.T))


@pytest.mark.parametrize("search", [0, 1])
@pytest.mark.parametrize("map_level,periodic", [(5, False), (7, False), (7, True)])
def test_value_records_bit_identical(ot, deep, search, map_level, periodic):
    """Uniform points (most of them in coarse leaves, which get value records) give the same
    results with the records (hot level set by the point count, and capped at 1, 3 and 4) and
    without them, in the caller's order and Morton-ordered, over two replays, and match the
    oracle (periodic cube too: the octant's neighbour wraps); points outside the cube get no
    host and NaN values either way."""
    import torch
    sph, ko, lo, _, field = deep
    t = ot.ot_octree_build(sph, 3, 9)
    ot.ot_octree_set_map_level(t, map_level)
    if search == 1:
        ot.ot_index_train(t, root=ot.OT_ROOT_MLP, n_leaf_models=4096, epochs=1, batch=16384)
    if periodic:
        ot.ot_octree_set_periodic(t, True)
    ot.ot_octree_build_mates(t, True)
    rng = np.random.default_rng(77)
    P = np.concatenate([rng.uniform(0, 1, (300000, 3)), face_points(ko, lo, rng, 4000),
                        np.array([[1.0, 0.5, 0.5], [0.5, -1e-9, 0.5], [np.nan, 0.5, 0.5]])])
    x, y, z = pts(P.T)
    f32 = dev(field.astype(np.float32))
    outs = []
    shapes = [dict(tri_records=-1), dict(), dict(tile=8, tri_tile=4), dict(order_level=6)]
    shapes += [dict(tri_records=k) for k in (1, 3, 4)]
    for lp in shapes:
        up = torch.full((3, P.shape[0]), 7.0, device="cuda")
        hp = torch.full((P.shape[0],), -5, dtype=torch.int32, device="cuda")
        b = ot.ot_batch_create(t, [dict(kernel=ot.OT_TRILINEAR, x=x, y=y, z=z, u=up, host=hp)], f32, search=search,
                               launch=lp)
        ot.ot_batch_run(b)
        ot.ot_batch_run(b)  # a second replay: means and records recomputed over the same buffers
        torch.cuda.synchronize()
        ot.ot_batch_destroy(b)
        outs.append((up, hp))
    for (up, hp), lp in zip(outs[1:], shapes[1:]):
        assert torch.equal(hp, outs[0][1]), lp
        assert torch.equal(up.isnan(), outs[0][0].isnan()), lp
        assert torch.equal(torch.nan_to_num(up, nan=0.0), torch.nan_to_num(outs[0][0], nan=0.0)), lp
    hp = outs[1][1].cpu().numpy()
    href = oracle.locate_ub(ko, lo, *P.T)
    assert np.array_equal(hp, href)
    inside = href >= 0
    assert inside.sum() == P.shape[0] - 3
    ref = oracle.interp_trilinear(ko, lo, field.astype(np.float32).astype(np.float64), *P[inside].T, href[inside],
                                  periodic=periodic)
    for up, _ in outs:
        assert rel_err(up.cpu().numpy()[:, inside], ref) <= TOL32
    assert torch.isnan(outs[1][0][:, ~torch.as_tensor(inside, device="cuda")]).all()


def test_uniform_and_random_trees(ot):
    import torch
    from paper_2605_20565_gb300 import synth
    rng = np.random.default_rng(77)
    cases = [(np.zeros((0, 5)), 4, 4), (np.zeros((0, 5)), 0, 0)]
    for _ in range(3):
        k = int(rng.integers(1, 4))
        sph = np.column_stack([rng.uniform(0.1, 0.9, (k, 3)), rng.uniform(0.05, 0.3, k), rng.uniform(0.0, 0.05, k)])
        cases.append((sph, int(rng.integers(1, 3)), int(rng.integers(4, 7))))
    for sph, lmin, lmax in cases:
        ko, lo = oracle.octree_build(sph, lmin, lmax)
        t = ot.ot_octree_build(sph, lmin, lmax)
        field = synth.sin_field(oracle.leaf_centres(ko, lo)).astype(np.float32)
        P = face_points(ko, lo, rng, 1500)
        x, y, z = pts(P.T)
        (u,), (um,) = both(ot, t, lambda: (ot.ot_interpolate(t, ot.OT_TRILINEAR, x, y, z, dev(field)),))
        assert torch.equal(u, um), (lmin, lmax)
        href = oracle.locate_ub(ko, lo, *P.T)
        ref = oracle.interp_trilinear(ko, lo, field.astype(np.float64), *P.T, href)
        assert rel_err(um.cpu().numpy(), ref) <= TOL32, (lmin, lmax)


def test_periodic_table_follows_the_setting(ot, deep):
    import torch
    sph, ko, lo, P, field = deep
    t = ot.ot_octree_build(sph, 3, 9)
    rng = np.random.default_rng(23)
    Q = np.concatenate([P[:3000], rng.uniform(0, 0.02, (800, 3)), 1.0 - rng.uniform(1e-9, 0.02, (800, 3))])
    f32 = field.astype(np.float32)
    x, y, z = pts(Q.T)
    host = oracle.locate_ub(ko, lo, *Q.T)
    ot.ot_octree_build_mates(t, True)
    for periodic in (True, False, True):
        ot.ot_octree_set_periodic(t, periodic)  # rebuilds the table
        assert ot.ot_octree_has_mates(t)
        um = ot.ot_interpolate(t, ot.OT_TRILINEAR, x, y, z, dev(f32))
        ref = oracle.interp_trilinear(ko, lo, f32.astype(np.float64), *Q.T, host, periodic=periodic)
        assert rel_err(um.cpu().numpy(), ref) <= TOL32, periodic
    ot.ot_octree_build_mates(t, False)
    u = ot.ot_interpolate(t, ot.OT_TRILINEAR, x, y, z, dev(f32))
    assert torch.equal(u, um)


def test_argument_errors(ot, deep):
    sph, ko, lo, P, field = deep
    t = ot.ot_octree_build(sph, 3, 9)
    with pytest.raises(Exception):
        ot.ot_octree_build_mates(t, 2)
    ot.ot_octree_build_mates(t, False)  # freeing an absent table is a no-op
    assert not ot.ot_octree_has_mates(t)


def test_autotune_with_table(ot):
    """With the table the two launches are tuned one after the other (16 delta shapes, 24
    trilinear shapes) and the chosen shape keeps the results."""
    import torch
    from paper_2605_20565_gb300 import synth
    w = synth.tiny()
    tree = ot.ot_octree_build(w.spheres, w.lmin, w.lmax)
    ot.ot_octree_build_mates(tree, True)
    cen = ot.ot_octree_centres(tree).cpu().numpy()
    field = dev(synth.sin_field(cen.T).astype(np.float32))
    mx, my, mz = pts(w.markers)
    px, py, pz = pts(w.particles)
    um = torch.empty((3, w.markers.shape[1]), device="cuda")
    up = torch.empty((3, w.particles.shape[1]), device="cuda")
    groups = [dict(kernel=ot.OT_PESKIN4, x=mx, y=my, z=mz, u=um), dict(kernel=ot.OT_TRILINEAR, x=px, y=py, z=pz, u=up)]
    ref_m = ot.ot_interpolate(tree, ot.OT_PESKIN4, mx, my, mz, field)
    ref_p = ot.ot_interpolate(tree, ot.OT_TRILINEAR, px, py, pz, field)
    r = ot.ot_batch_autotune(tree, groups, field, search=ot.OT_BINARY, tune_map_level=True, reps=1)
    assert r["tried"] == 16 + 24 and r["map_level"] == 5 and r["ms"] > 0
    lp = r["launch"]
    assert lp["tri_tile"] in (2, 4, 8) and lp["order_level"] in (0, 8)
    assert lp["tri_blocks_per_sm"] in [k * 256 // lp["block"] for k in (1, 2, 3, 4)]
    b = ot.ot_batch_create(tree, groups, field, launch=lp)
    ot.ot_batch_run(b)
    torch.cuda.synchronize()
    assert torch.equal(um, ref_m) and torch.equal(up, ref_p)


def test_table_in_caller_buffer(ot, deep):
    """The table built in a caller buffer gives the same results; the buffer outlives the octree
    and serves the next one; short or misaligned buffers are refused."""
    import torch
    sph, ko, lo, P, field = deep
    f32 = dev(field.astype(np.float32))
    x, y, z = pts(P.T)
    t = ot.ot_octree_build(sph, 3, 9)
    ref = ot.ot_interpolate(t, ot.OT_TRILINEAR, x, y, z, f32)
    need = ot.ot_octree_mates_bytes(t)
    assert need == 256 * ko.size + 128 * (ko.size // 8 + 1)  # level-mate rows, then parent-block rows
    buf = torch.empty(need + 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(ot.OtError):
        ot.ot_octree_build_mates_in(t, buf[: need - 16])
    with pytest.raises(ot.OtError):
        ot.ot_octree_build_mates_in(t, buf[8: need + 8])
    assert not ot.ot_octree_has_mates(t)
    ot.ot_octree_build_mates_in(t, buf)
    assert ot.ot_octree_has_mates(t)
    assert torch.equal(ot.ot_interpolate(t, ot.OT_TRILINEAR, x, y, z, f32), ref)
    del t  # the caller's buffer stays allocated
    t2 = ot.ot_octree_build(sph, 3, 9)
    ot.ot_octree_build_mates(t2, True)  # a library-owned table first, then replaced
    ot.ot_octree_build_mates_in(t2, buf)
    assert torch.equal(ot.ot_interpolate(t2, ot.OT_TRILINEAR, x, y, z, f32), ref)
    ot.ot_octree_build_mates(t2, False)
    assert not ot.ot_octree_has_mates(t2)


@pytest.mark.parametrize("kernel", [2, 3])
@pytest.mark.parametrize("periodic", [False, True])
def test_parent_block_table_delta_paths(ot, kernel, periodic):
    """Delta-kernel interpolation and sorted spreading read the parent-block table built with
    the level-mate table: identical bits with and without it, and the oracle's values --
    markers on a refined sphere, across the cube's faces (periodic), and in cells whose
    stencils leave the finest level."""
    import torch
    from paper_2605_20565_gb300 import synth
    sph = np.array([[0.5, 0.5, 0.5, 0.2, 0.06], [0.05, 0.95, 0.5, 0.1, 0.06]])
    ko, lo = oracle.octree_build(sph, 3, 7)
    t = ot.ot_octree_build(sph, 3, 7)
    if periodic:
        ot.ot_octree_set_periodic(t, True)
    rng = np.random.default_rng(8)
    d = rng.normal(size=(3, 3000))
    X = np.concatenate([np.array([[0.5], [0.5], [0.5]]) + 0.2 * d / np.linalg.norm(d, axis=0),
                        np.array([[0.05], [0.95], [0.5]]) + 0.1 * d / np.linalg.norm(d, axis=0),
                        rng.uniform(0, 1, (3, 500))], 1)
    X = np.mod(X, 1.0)
    X = X[:, np.all((X >= 0) & (X < 1), axis=0)]
    field = synth.sin_field(oracle.leaf_centres(ko, lo)).astype(np.float32)
    F = rng.normal(size=(3, X.shape[1])).astype(np.float32)
    x, y, z = pts(X)

    def run():
        u = ot.ot_interpolate(t, kernel, x, y, z, dev(field))
        f = torch.zeros((ko.size, 4), dtype=torch.float32, device="cuda")
        ot.ot_spread(t, kernel, ot.OT_SORTED, x, y, z, dev(F), f)
        fa = torch.zeros((ko.size, 4), dtype=torch.float32, device="cuda")
        ot.ot_spread(t, kernel, ot.OT_ATOMIC, x, y, z, dev(F), fa)
        return u, f, fa

    (u, f, fa), (um, fm, fam) = both(ot, t, run)
    assert torch.equal(u, um) and torch.equal(f, fm)
    assert float((fa - fam).abs().max()) <= 1e-5 * float(f.abs().max())
    ref, _ = oracle.interp_delta(ko, lo, 7, kernel, field.astype(np.float64), *X, periodic=periodic)
    ok = ~np.isnan(ref).any(axis=0)
    assert rel_err(um.cpu().numpy()[:, ok], ref[:, ok]) <= TOL32
    fref, _ = oracle.spread_delta(ko, lo, 7, kernel, *X, F.astype(np.float64), periodic=periodic)
    assert rel_err(fm.cpu().numpy()[:, :3], fref[:, :3]) <= TOL32
