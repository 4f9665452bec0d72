"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded
inputs.  Host indices and octree leaves are compared bit for bit; FP32 values within 1e-5 of
max|reference| (the tolerance stated for this path), FP64 values within 1e-12."""
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


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def pts(a):
    return [dev(np.ascontiguousarray(a[d], dtype=np.float64)) for d in range(3)]


def leaves_np(ot, tree):
    k, l = ot.ot_octree_copy_leaves(tree)
    return k.cpu().numpy().view(np.uint64), l.cpu().numpy()


def rel_err(a, ref):
    scale = max(np.abs(ref).max(), 1e-300)
    return float(np.abs(a - ref).max() / scale)


@pytest.fixture(scope="module")
def tiny(ot):
    from paper_2605_20565_gb300 import synth
    w = synth.tiny()
    ko, lo = oracle.octree_build(w.spheres, w.lmin, w.lmax)
    tree = ot.ot_octree_build(w.spheres, w.lmin, w.lmax)
    return w, ko, lo, tree


# ---------------------------------------------------------------------------------------
# Octree construction
# ---------------------------------------------------------------------------------------

def test_tiny_octree_bit_exact(ot, tiny):
    w, ko, lo, tree = tiny
    k, l = leaves_np(ot, tree)
    assert np.array_equal(k, ko) and np.array_equal(l, lo)
    assert ot.ot_octree_info(tree) == (ko.size, w.lmin, w.lmax)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("full", [1, 0])
def test_random_octrees_bit_exact(ot, seed, full):
    rng = np.random.default_rng(1000 + seed)
    lmin = int(rng.integers(0, 4))
    lmax = int(rng.integers(lmin, 8))
    ns = int(rng.integers(0, 6))
    sph = np.column_stack([rng.uniform(0.0, 1.0, (ns, 3)), rng.uniform(0.0, 0.3, ns), rng.uniform(0.0, 0.1, ns)])
    ko, lo = oracle.octree_build(sph, lmin, lmax, full)
    tree = ot.ot_octree_build(sph, lmin, lmax, full)
    k, l = leaves_np(ot, tree)
    assert np.array_equal(k, ko) and np.array_equal(l, lo)
    # every level-map level (subtree descriptors of every depth, and the search fallback)
    # locates and interpolates exactly as the oracle
    P = special_points(ko, lo, rng, 3000)
    ref = oracle.locate_ub(ko, lo, *P.T)
    Pi = P[ref >= 0]
    f32 = rng.normal(size=(ko.size, 4)).astype(np.float32)
    uref = oracle.interp_trilinear(ko, lo, f32.astype(np.float64), *Pi.T, ref[ref >= 0])
    for L in range(0, min(lmax, 8) + 1):
        ot.ot_octree_set_map_level(tree, L)
        assert np.array_equal(ot.ot_locate(tree, *pts(P.T)).cpu().numpy(), ref), L
        u = ot.ot_interpolate(tree, ot.OT_TRILINEAR, *pts(Pi.T), dev(f32)).cpu().numpy()
        assert rel_err(u, uref) <= TOL32, L


def test_uniform_and_single_leaf_trees(ot):
    for lev in (0, 1, 3):
        ko, lo = oracle.octree_build(np.zeros((0, 5)), lev, lev)
        tree = ot.ot_octree_build(np.zeros((0, 5)), lev, lev)
        k, l = leaves_np(ot, tree)
        assert np.array_equal(k, ko) and np.array_equal(l, lo)


def test_from_leaves_validation(ot, tiny, torch_mod):
    torch = torch_mod
    w, ko, lo, tree = tiny
    kt = dev(ko.view(np.int64))
    lt = dev(lo)
    t2 = ot.ot_octree_from_leaves(kt, lt)
    assert ot.ot_octree_info(t2)[0] == ko.size
    # unsorted
    bad = ko.copy()
    bad[[10, 11]] = bad[[11, 10]]
    with pytest.raises(ot.OtError) as e:
        ot.ot_octree_from_leaves(dev(bad.view(np.int64)), lt)
    assert e.value.status == -4
    # a gap (one leaf removed)
    with pytest.raises(ot.OtError) as e:
        ot.ot_octree_from_leaves(dev(np.delete(ko, 5).view(np.int64)), dev(np.delete(lo, 5)))
    assert e.value.status == -4
    # unbalanced: level-1 octants next to a block refined to level 3
    keys, levels = [], []
    for c in range(8):
        if c == 0:
            for g in range(64):
                keys.append(g << (3 * 18))
                levels.append(3)
        else:
            keys.append(c << (3 * 20))
            levels.append(1)
    with pytest.raises(ot.OtError) as e:
        ot.ot_octree_from_leaves(dev(np.array(keys, np.uint64).view(np.int64)), dev(np.array(levels, np.uint8)))
    assert e.value.status == -5
    del torch


# ---------------------------------------------------------------------------------------
# Host-cell search
# ---------------------------------------------------------------------------------------

def special_points(ko, lo, rng, n_rand):
    cen = oracle.leaf_centres(ko, lo)
    h = 2.0 ** -lo.astype(np.float64)
    anchors = cen - 0.5 * h[:, None]
    P = np.concatenate([rng.uniform(0, 1, (n_rand, 3)), anchors, cen,
                        np.array([[1.0, 0.5, 0.5], [-1e-300, 0.5, 0.5], [np.nan, 0.5, 0.5],
                                  [np.nextafter(1.0, 0.0)] * 3, [0.0, 0.0, 0.0], [-0.0, 0.5, 0.5]])])
    return P


@pytest.mark.parametrize("map_level", [0, 2, 3, 5])
def test_level_map_levels(ot, tiny, tiny_fields, map_level):
    """Every level of the level map gives the same hosts and values: a covered cell answers from
    the map, any other point is searched among its cell's leaves."""
    w, ko, lo, tree = tiny
    t2 = ot.ot_octree_build(w.spheres, w.lmin, w.lmax)
    ot.ot_octree_set_map_level(t2, map_level)
    P = special_points(ko, lo, np.random.default_rng(77), 4000)
    h = ot.ot_locate(t2, *pts(P.T))
    assert np.array_equal(h.cpu().numpy(), oracle.locate_ub(ko, lo, *P.T))
    f32 = tiny_fields["sin"].astype(np.float32)
    Pi = P[:-6]
    u = ot.ot_interpolate(t2, ot.OT_TRILINEAR, *pts(Pi.T), dev(f32)).cpu().numpy()
    href = oracle.locate_ub(ko, lo, *Pi.T)
    ref = oracle.interp_trilinear(ko, lo, f32.astype(np.float64), *Pi.T, href)
    assert rel_err(u, ref) <= TOL32
    um = ot.ot_interpolate(t2, 2, *pts(w.markers), dev(f32)).cpu().numpy()
    refm, _ = oracle.interp_delta(ko, lo, w.lmax, 2, f32.astype(np.float64), *w.markers)
    assert rel_err(um, refm) <= TOL32
    ot.ot_index_train(t2, root=ot.OT_ROOT_MLP, n_leaf_models=512, n_mid_models=32, epochs=1, batch=4096)
    hl = ot.ot_locate(t2, *pts(P.T), search=ot.OT_LEARNED)
    assert np.array_equal(hl.cpu().numpy(), h.cpu().numpy())


@pytest.mark.parametrize("n", [0, 1, 31, 33, 1007])
def test_locate_binary_ragged(ot, tiny, n):
    w, ko, lo, tree = tiny
    rng = np.random.default_rng(n)
    P = rng.uniform(0, 1, (n, 3))
    x, y, z = pts(P.T) if n else [dev(np.zeros(0))] * 3
    h = ot.ot_locate(tree, x, y, z)
    ref = oracle.locate_ub(ko, lo, *P.T) if n else np.zeros(0, np.int32)
    assert np.array_equal(h.cpu().numpy(), ref)


def test_locate_special_points(ot, tiny, torch_mod):
    torch = torch_mod
    w, ko, lo, tree = tiny
    P = special_points(ko, lo, np.random.default_rng(5), 3000)
    ref = oracle.locate_ub(ko, lo, *P.T)
    assert np.array_equal(ref, oracle.locate_brute(ko, lo, *P.T))
    miss = torch.zeros(1, dtype=torch.int64, device="cuda")
    h = ot.ot_locate(tree, *pts(P.T), n_miss=miss)
    assert np.array_equal(h.cpu().numpy(), ref)
    assert int(miss.item()) == int((ref < 0).sum()) == 3
    assert ot.ot_last_error(tree) & ot.OT_DEV_OUTSIDE


@pytest.mark.parametrize("root,mid", [(0, 0), (1, 0), (1, 64)])
def test_learned_locate_bit_exact(ot, root, mid):
    from paper_2605_20565_gb300 import synth
    w = synth.single_bubble(n_markers=2000, n_particles=200_000)
    w.lmin, w.lmax = 4, 8
    sph = w.spheres.copy()
    sph[:, 4] = 0.1
    ko, lo = oracle.octree_build(sph, 4, 8)
    tree = ot.ot_octree_build(sph, 4, 8)
    ot.ot_index_train(tree, root=root, n_leaf_models=1024 if not mid else 8192, n_mid_models=mid, epochs=2,
                      batch=8192, lr=1e-3, seed=7)
    P = special_points(ko, lo, np.random.default_rng(9), 20000)
    P = np.concatenate([P, w.particles.T])
    x, y, z = pts(P.T)
    hb = ot.ot_locate(tree, x, y, z, search=ot.OT_BINARY)
    hl = ot.ot_locate(tree, x, y, z, search=ot.OT_LEARNED)
    ref = oracle.locate_ub(ko, lo, *P.T)
    assert np.array_equal(hb.cpu().numpy(), ref)
    assert np.array_equal(hl.cpu().numpy(), ref)
    # every stored key (the leaf anchors) is answered inside its window: no fallback
    cen = oracle.leaf_centres(ko, lo)
    anchors = cen - 0.5 * (2.0 ** -lo.astype(np.float64))[:, None]
    ot.ot_index_get_stats(tree, reset=True)
    ha = ot.ot_locate(tree, *pts(anchors.T), search=ot.OT_LEARNED)
    assert np.array_equal(ha.cpu().numpy(), np.arange(ko.size, dtype=np.int32))
    st = ot.ot_index_get_stats(tree)
    assert st["fallbacks"] == 0
    assert st["mean_window"] < ko.size / 8


# ---------------------------------------------------------------------------------------
# Interpolation
# ---------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def tiny_fields(tiny):
    from paper_2605_20565_gb300 import synth
    w, ko, lo, tree = tiny
    cen = oracle.leaf_centres(ko, lo)
    return {"sin": synth.sin_field(cen), "linear": synth.linear_field(cen)}


@pytest.mark.parametrize("fname", ["sin", "linear"])
@pytest.mark.parametrize("search", [0, 1])
def test_trilinear_f32(ot, tiny, tiny_fields, fname, search, torch_mod):
    torch = torch_mod
    w, ko, lo, tree = tiny
    if search == 1:
        ot.ot_index_train(tree, root=ot.OT_ROOT_LINEAR, n_leaf_models=128)
    P = special_points(ko, lo, np.random.default_rng(3), 5000)[:-6]  # inside the cube
    f32 = tiny_fields[fname].astype(np.float32)
    field = dev(f32)
    hout = torch.empty(P.shape[0], dtype=torch.int32, device="cuda")
    u = ot.ot_interpolate(tree, ot.OT_TRILINEAR, *pts(P.T), field, search=search, host_out=hout)
    href = oracle.locate_ub(ko, lo, *P.T)
    ref = oracle.interp_trilinear(ko, lo, f32.astype(np.float64), *P.T, href)
    assert np.array_equal(hout.cpu().numpy(), href)
    assert rel_err(u.cpu().numpy(), ref) <= TOL32
    # with given host indices
    u2 = ot.ot_interpolate(tree, ot.OT_TRILINEAR, *pts(P.T), field, host_in=hout)
    assert torch.equal(u, u2)


def test_trilinear_f64_and_outside(ot, tiny, tiny_fields):
    w, ko, lo, tree = tiny
    P = special_points(ko, lo, np.random.default_rng(4), 5000)
    field = tiny_fields["sin"]
    u = ot.ot_interpolate_f64(tree, ot.OT_TRILINEAR, *pts(P.T), dev(field)).cpu().numpy()
    href = oracle.locate_ub(ko, lo, *P.T)
    ref = oracle.interp_trilinear(ko, lo, field, *P.T, href)
    inside = href >= 0
    assert np.all(np.isnan(u[:, ~inside]))
    assert rel_err(u[:, inside], ref[:, inside]) <= TOL64


@pytest.mark.parametrize("kernel", [2, 3])
@pytest.mark.parametrize("search", [0, 1])
def test_delta_interp(ot, tiny, tiny_fields, kernel, search, torch_mod):
    torch = torch_mod
    w, ko, lo, tree = tiny
    if search == 1:
        ot.ot_index_train(tree, root=ot.OT_ROOT_LINEAR, n_leaf_models=128)
    ot.ot_last_error(tree)  # clear bits left by earlier tests
    X = w.markers
    for fname in ("sin", "linear"):
        f64 = tiny_fields[fname]
        f32 = f64.astype(np.float32)
        hout = torch.empty(X.shape[1], dtype=torch.int32, device="cuda")
        u = ot.ot_interpolate(tree, kernel, *pts(X), dev(f32), search=search, host_out=hout)
        ref, bad = oracle.interp_delta(ko, lo, w.lmax, kernel, f32.astype(np.float64), *X)
        assert bad == 0
        assert rel_err(u.cpu().numpy(), ref) <= TOL32
        assert np.array_equal(hout.cpu().numpy(), oracle.locate_ub(ko, lo, *X))
        u64 = ot.ot_interpolate_f64(tree, kernel, *pts(X), dev(f64), search=search)
        ref64, _ = oracle.interp_delta(ko, lo, w.lmax, kernel, f64, *X)
        assert rel_err(u64.cpu().numpy(), ref64) <= TOL64
    assert ot.ot_last_error(tree) & (ot.OT_DEV_STENCIL | ot.OT_DEV_OUTSIDE) == 0


def test_delta_stencil_errors_match_oracle(ot, tiny, tiny_fields):
    w, ko, lo, tree = tiny
    ot.ot_last_error(tree)
    P = np.array([[0.01, 0.99, 0.5], [0.01, 0.5, 0.5], [0.5, 0.3005, 0.5], [0.5, 0.5, 0.5]]).T.copy()
    f64 = tiny_fields["sin"]
    u = ot.ot_interpolate_f64(tree, 2, *pts(P), dev(f64))
    ref, bad = oracle.interp_delta(ko, lo, w.lmax, 2, f64, *P)
    assert bad > 0
    assert rel_err(u.cpu().numpy(), ref) <= TOL64
    assert ot.ot_last_error(tree) & ot.OT_DEV_STENCIL


# ---------------------------------------------------------------------------------------
# Spreading
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [2, 3])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("with_dv", [False, True])
def test_spread(ot, tiny, kernel, mode, with_dv, torch_mod):
    torch = torch_mod
    w, ko, lo, tree = tiny
    rng = np.random.default_rng(21)
    X = w.markers
    n = X.shape[1]
    F = rng.normal(size=(3, n)).astype(np.float32)
    h3 = 2.0 ** (-3 * w.lmax)
    dV = (rng.uniform(0.5, 2.0, n) * h3).astype(np.float32) if with_dv else None
    f = torch.zeros((ko.size, 4), dtype=torch.float32, device="cuda")
    ot.ot_spread(tree, kernel, mode, *pts(X), dev(F), f, dV=dev(dV) if with_dv else None)
    ref, bad = oracle.spread_delta(ko, lo, w.lmax, kernel, *X, F.astype(np.float64),
                                   dV.astype(np.float64) if with_dv else None)
    assert bad == 0
    fn = f.cpu().numpy()
    assert rel_err(fn[:, :3], ref[:, :3]) <= TOL32
    assert np.all(fn[:, 3] == 0)
    # f64
    f64 = torch.zeros((ko.size, 4), dtype=torch.float64, device="cuda")
    ot.ot_spread_f64(tree, kernel, mode, *pts(X), dev(F.astype(np.float64)), f64,
                     dV=dev(dV.astype(np.float64)) if with_dv else None)
    assert rel_err(f64.cpu().numpy()[:, :3], ref[:, :3]) <= TOL64


def test_sorted_spread_is_deterministic_and_accumulates(ot, tiny, torch_mod):
    torch = torch_mod
    w, ko, lo, tree = tiny
    rng = np.random.default_rng(22)
    X = w.markers
    F = dev(rng.normal(size=(3, X.shape[1])).astype(np.float32))
    x, y, z = pts(X)
    outs = []
    for _ in range(10):
        f = torch.zeros((ko.size, 4), dtype=torch.float32, device="cuda")
        ot.ot_spread(tree, 2, ot.OT_SORTED, x, y, z, F, f)
        outs.append(f)
    for o in outs[1:]:
        assert torch.equal(o.view(torch.int32), outs[0].view(torch.int32))
    f = outs[0].clone()
    ot.ot_spread(tree, 2, ot.OT_SORTED, x, y, z, F, f)
    assert torch.equal(f, 2 * outs[0])
    with pytest.raises(ot.OtError):
        ot.ot_spread(tree, 2, ot.OT_SORTED, x, y, z, F, f,
                     workspace=torch.empty(64, dtype=torch.uint8, device="cuda"))


def test_adjoint_identity_on_device(ot, tiny, torch_mod):
    """<I u, F>_L = <u, S F>_E with h^3 weights, both sides computed by the CUDA path (FP64)."""
    torch = torch_mod
    w, ko, lo, tree = tiny
    rng = np.random.default_rng(23)
    X = w.markers
    n = X.shape[1]
    F = rng.normal(size=(3, n))
    uf = np.zeros((ko.size, 4))
    uf[:, :3] = rng.normal(size=(ko.size, 3))
    Iu = ot.ot_interpolate_f64(tree, 2, *pts(X), dev(uf)).cpu().numpy()
    f = torch.zeros((ko.size, 4), dtype=torch.float64, device="cuda")
    ot.ot_spread_f64(tree, 2, ot.OT_SORTED, *pts(X), dev(F), f)
    h3 = 2.0 ** (-3 * w.lmax)
    lhs = float((Iu * F).sum() * h3)
    rhs = float((uf[:, :3] * f.cpu().numpy()[:, :3]).sum() * h3)
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))


# ---------------------------------------------------------------------------------------
# Learned-index network gradient
# ---------------------------------------------------------------------------------------

def test_mlp_gradient_matches_oracle(ot, torch_mod):
    torch = torch_mod
    rng = np.random.default_rng(5)
    prm = rng.normal(scale=0.5, size=97).astype(np.float32)
    x = rng.uniform(0, 1, 4096).astype(np.float32)
    t = np.sort(rng.uniform(0, 1, 4096)).astype(np.float32)
    g, loss = ot.ot_index_mlp_grad(dev(prm), dev(x), dev(t))
    lref, gref = oracle.mlp_loss_grad(prm.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss.item() - lref) <= 1e-4 * abs(lref)
    assert np.abs(g.cpu().numpy() - gref).max() <= 1e-3 * np.abs(gref).max()
    del torch


# ---------------------------------------------------------------------------------------
# Batched persistent launch
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("search", [0, 1])
def test_batch_matches_single_ops(ot, tiny, tiny_fields, search, torch_mod):
    torch = torch_mod
    w, ko, lo, tree = tiny
    ot.ot_index_train(tree, root=ot.OT_ROOT_MLP, n_leaf_models=256, epochs=2, batch=4096)
    field = dev(tiny_fields["sin"].astype(np.float32))
    X = w.markers
    P = w.particles
    mx, my, mz = pts(X)
    px, py, pz = pts(P)
    X3 = np.ascontiguousarray(X[:, :333])
    gx, gy, gz = pts(X3)
    um = torch.full((3, X.shape[1]), 7.0, device="cuda")
    up = torch.full((3, P.shape[1]), 7.0, device="cuda")
    ur = torch.full((3, X3.shape[1]), 7.0, device="cuda")
    hp = torch.empty(P.shape[1], dtype=torch.int32, device="cuda")
    b = ot.ot_batch_create(tree, [dict(kernel=2, x=mx, y=my, z=mz, u=um),
                                  dict(kernel=1, x=px, y=py, z=pz, u=up, host=hp),
                                  dict(kernel=3, x=gx, y=gy, z=gz, u=ur)], field, search=search,
                           launch=dict(block=128, tile=2))
    for _ in range(2):
        ot.ot_batch_run(b)
    torch.cuda.synchronize()
    assert torch.equal(um, ot.ot_interpolate(tree, 2, mx, my, mz, field, search=search))
    assert torch.equal(up, ot.ot_interpolate(tree, 1, px, py, pz, field, search=search))
    assert torch.equal(ur, ot.ot_interpolate(tree, 3, gx, gy, gz, field, search=search))
    assert np.array_equal(hp.cpu().numpy(), oracle.locate_ub(ko, lo, *P))


@pytest.mark.parametrize("order_level", [5, 8])
def test_ordered_batch_gives_identical_results(ot, deep, order_level, torch_mod):
    """Points interpolated in Morton order of their cells inside the graph, results written
    back in the caller's order: the same values and hosts bit for bit."""
    torch = torch_mod
    sph, ko, lo, P, field = deep
    t = ot.ot_octree_build(sph, 3, 9)
    f32 = dev(field.astype(np.float32))
    x, y, z = pts(P.T)
    outs = []
    for lv in (0, order_level):
        u = torch.full((3, P.shape[0]), 7.0, device="cuda")
        h = torch.full((P.shape[0],), -5, dtype=torch.int32, device="cuda")
        b = ot.ot_batch_create(t, [dict(kernel=ot.OT_TRILINEAR, x=x, y=y, z=z, u=u, host=h)], f32,
                               launch=dict(order_level=lv))
        ot.ot_batch_run(b)
        ot.ot_batch_run(b)
        torch.cuda.synchronize()
        outs.append((u, h))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[1][1].cpu().numpy(), oracle.locate_ub(ko, lo, *P.T))


# ---------------------------------------------------------------------------------------
# Advection step
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1000, 1001])  # the 4-particle vector kernel, and the scalar one
def test_advect_ab2_matches_oracle(ot, torch_mod, n):
    torch = torch_mod
    rng = np.random.default_rng(31)
    x = rng.uniform(0.2, 0.8, (3, n))
    v = rng.normal(scale=0.1, size=(3, n)).astype(np.float32)
    u = rng.normal(scale=0.1, size=(3, n)).astype(np.float32)
    st = {"x": x.copy(), "v": v.astype(np.float64), "a_prev": np.zeros((3, n)), "v_prev": np.zeros((3, n))}
    dx, dv = dev(x), dev(v)
    da, dvp = torch.zeros_like(dv), torch.zeros_like(dv)
    for step in range(3):
        oracle.advect_ab2(st, u.astype(np.float64), 0.05, 2.0, 1e-3, step == 0)
        ot.ot_advect_ab2(dx, dv, da, dvp, dev(u), 0.05, 2.0, 1e-3, step == 0)
    assert rel_err(dv.cpu().numpy(), st["v"]) <= TOL32
    assert np.abs(dx.cpu().numpy() - st["x"]).max() <= 1e-9


def test_advect_vector_and_scalar_kernels_agree(ot, torch_mod):
    """The 4-particle kernel (aligned planes) and the scalar one (planes 4 bytes off) give the
    same bits, with the drag law on and positions wrapping at every face."""
    torch = torch_mod
    rng = np.random.default_rng(32)
    n = 4096
    x0 = np.concatenate([rng.uniform(0, 1e-4, (3, n // 2)), 1.0 - rng.uniform(1e-12, 1e-4, (3, n // 2))], 1)
    v0 = rng.normal(scale=0.5, size=(3, n)).astype(np.float32)
    u0 = rng.normal(scale=0.5, size=(3, n)).astype(np.float32)
    outs = []
    for off in (0, 1):
        def buf(a, dtype):
            t = torch.zeros(3 * n + off, dtype=dtype, device="cuda")
            t[off:] = torch.as_tensor(np.ascontiguousarray(a).reshape(-1), dtype=dtype)
            return t[off:].view(3, n)
        x, v = buf(x0, torch.float64), buf(v0, torch.float32)
        ap, vp, u = buf(np.zeros((3, n)), torch.float32), buf(np.zeros((3, n)), torch.float32), buf(u0, torch.float32)
        for step in range(3):
            ot.ot_advect_ab2(x, v, ap, vp, u, 0.05, 2.0, 1e-3, step == 0, periodic=True)
        outs.append([t.clone() for t in (x, v, ap, vp)])
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    assert bool(((outs[0][0] >= 0) & (outs[0][0] < 1)).all())


@pytest.fixture(scope="module")
def deep(ot):
    """Levels 3-9 around two small spheres (~294k leaves): host leaves of levels 7-9 have refined
    level-mates both inside the pyramid of cell means (level <= 7) and below it."""
    sph = np.array([[0.53, 0.47, 0.51, 0.05, 0.02], [0.2, 0.7, 0.3, 0.03, 0.015]])
    ko, lo = oracle.octree_build(sph, 3, 9)
    rng = np.random.default_rng(91)
    d = rng.normal(size=(30000, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    which = rng.integers(0, 2, 30000)
    rad = sph[which, 3] + rng.uniform(-3, 3, 30000) * sph[which, 4]
    P = np.concatenate([sph[which, :3] + d * rad[:, None], rng.uniform(0, 1, (5000, 3))])
    P = P[np.all((P >= 0) & (P < 1), axis=1)]
    from paper_2605_20565_gb300 import synth
    field = synth.sin_field(oracle.leaf_centres(ko, lo))
    return sph, ko, lo, P, field


@pytest.mark.parametrize("map_level", [-1, 0, 8])
def test_deep_tree_trilinear(ot, deep, map_level, torch_mod):
    sph, ko, lo, P, field = deep
    t = ot.ot_octree_build(sph, 3, 9)
    kt, lt = leaves_np(ot, t)
    assert np.array_equal(kt, ko) and np.array_equal(lt, lo)
    if map_level >= 0:
        ot.ot_octree_set_map_level(t, map_level)
    href = oracle.locate_ub(ko, lo, *P.T)
    f32 = field.astype(np.float32)
    ref32 = oracle.interp_trilinear(ko, lo, f32.astype(np.float64), *P.T, href)
    hout = torch_mod.empty(P.shape[0], dtype=torch_mod.int32, device="cuda")
    u = ot.ot_interpolate(t, ot.OT_TRILINEAR, *pts(P.T), dev(f32), host_out=hout).cpu().numpy()
    assert np.array_equal(hout.cpu().numpy(), href)
    assert rel_err(u, ref32) <= TOL32
    u64 = ot.ot_interpolate_f64(t, ot.OT_TRILINEAR, *pts(P.T), dev(field)).cpu().numpy()
    assert rel_err(u64, oracle.interp_trilinear(ko, lo, field, *P.T, href)) <= TOL64
    # the batched form (pyramid rebuilt inside the graph) gives the same values
    ot.ot_index_train(t, root=ot.OT_ROOT_MLP, n_leaf_models=4096, n_mid_models=64, epochs=1, batch=16384)
    for search in (0, 1):
        ub = torch_mod.empty((3, P.shape[0]), dtype=torch_mod.float32, device="cuda")
        x, y, z = pts(P.T)
        b = ot.ot_batch_create(t, [dict(kernel=ot.OT_TRILINEAR, x=x, y=y, z=z, u=ub)], dev(f32), search=search)
        ot.ot_batch_run(b)
        assert rel_err(ub.cpu().numpy(), ref32) <= TOL32
    assert ot.ot_last_error(t) & (ot.OT_DEV_OUTSIDE | ot.OT_DEV_STENCIL) == 0


# ---------------------------------------------------------------------------------------
# Multi-direct forcing (Sec. 2.2)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [2, 3])
@pytest.mark.parametrize("with_dv", [False, True])
def test_mdf_matches_oracle(ot, tiny, tiny_fields, kernel, with_dv, torch_mod):
    torch = torch_mod
    w, ko, lo, tree = tiny
    rng = np.random.default_rng(31)
    X = w.markers
    nm = X.shape[1]
    u_star = tiny_fields["sin"].astype(np.float32)
    U = (0.3 * rng.normal(size=(3, nm))).astype(np.float32)
    h3 = 2.0 ** (-3 * w.lmax)
    dV = (rng.uniform(0.5, 2.0, nm) * h3).astype(np.float32) if with_dv else None
    rho, dt, n_iter = 1.3, 0.7, 4
    u_ref, f_ref, slip_ref, bad = oracle.ibm_mdf(ko, lo, w.lmax, kernel, u_star.astype(np.float64), X,
                                                 U.astype(np.float64), rho, dt, n_iter,
                                                 dV=None if dV is None else dV.astype(np.float64))
    assert bad == 0
    u = dev(u_star)
    f, slip = ot.ot_ibm_mdf(tree, kernel, *pts(X), dev(U), u, rho, dt, n_iter,
                            dV=None if dV is None else dev(dV), slip=True)
    torch.cuda.synchronize()
    assert rel_err(u.cpu().numpy()[:, :3], u_ref[:, :3]) <= TOL32
    assert np.array_equal(u.cpu().numpy()[:, 3], u_star[:, 3])
    assert rel_err(f.cpu().numpy()[:, :3], f_ref[:, :3]) <= TOL32
    assert np.abs(slip.cpu().numpy() - slip_ref).max() <= 1e-5 * slip_ref.max()
    assert np.all(np.diff(slip_ref) < 0)
    # deterministic: a second run gives the same bits
    u2 = dev(u_star)
    f2, _ = ot.ot_ibm_mdf(tree, kernel, *pts(X), dev(U), u2, rho, dt, n_iter, dV=None if dV is None else dev(dV))
    assert torch.equal(u, u2) and torch.equal(f, f2)


@pytest.mark.parametrize("n,level", [(1, 8), (33, 19), (50000, 8), (50000, 5)])
def test_points_morton_order(ot, n, level, torch_mod):
    """The permutation equals a stable sort of the points' level-L Morton cell keys (an
    independent bit-loop encoder here)."""
    rng = np.random.default_rng(n + level)
    P = rng.uniform(0, 1, (3, n))
    if n > 40:
        P[:, :5] = P[:, 5:10]           # equal keys keep their input order
        P[0, 10] = 1.0                  # outside: last
    perm = ot.ot_points_morton_order(*pts(P), level=level).cpu().numpy()
    q = np.floor(np.clip(P, 0, 1) * 2.0 ** level).astype(np.uint64)
    key = np.zeros(n, np.uint64)
    for b in range(level):
        for d in range(3):
            key |= ((q[d] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + d)
    key[np.any((P < 0) | (P >= 1), axis=0)] = np.uint64((1 << (3 * level)) - 1)
    ref = np.argsort(key, kind="stable")
    assert np.array_equal(perm, ref)


def test_field_fourier_matches_modes(ot, deep):
    """The analytic leaf field (exact fixed-point phase, FP32 cosine) against the same modes
    evaluated in FP64 at the oracle's leaf centres."""
    from paper_2605_20565_gb300 import synth
    sph, ko, lo, P, _ = deep
    t = ot.ot_octree_build(sph, 3, 9)
    m = synth.fourier_modes(4)
    f = ot.ot_field_fourier(t, m.n, m.amp, m.phase).cpu().numpy()
    ref = synth.fourier_field(m, oracle.leaf_centres(ko, lo))
    assert np.abs(f[:, :3] - ref[:, :3]).max() <= 1e-6 * np.abs(ref).max()
    assert np.all(f[:, 3] == 0)


def test_body_sums_match_oracle(ot, deep, torch_mod):
    """Internal-fluid momenta of each body from trilinear velocities at its internal markers,
    and the IBM force and torque of surface-marker forces (Sec. 2.3), against the oracle."""
    torch = torch_mod
    from paper_2605_20565_gb300 import synth
    sph, ko, lo, P, field = deep
    t = ot.ot_octree_build(sph, 3, 9)
    h = 2.0 ** -9
    X, start = synth.internal_markers(sph[:, :3], 2.0 * sph[:, 3], h)
    f32 = field.astype(np.float32)
    u = ot.ot_interpolate(t, ot.OT_TRILINEAR, *pts(X), dev(f32))
    href = oracle.locate_ub(ko, lo, *X)
    uref = oracle.interp_trilinear(ko, lo, f32.astype(np.float64), *X, href)
    rho = 1.2
    d_start = torch.as_tensor(start, device="cuda")
    xb = torch.as_tensor(np.ascontiguousarray(sph[:, :3]), device="cuda")
    lin, ang = ot.ot_body_sums(*pts(X), u, d_start, xb, rho, w=h ** 3)
    lref, aref = oracle.body_sums(X, uref, start, sph[:, :3], rho, w=h ** 3)
    assert rel_err(lin.cpu().numpy(), lref) <= TOL32
    assert rel_err(ang.cpu().numpy(), aref) <= TOL32
    # surface forces with marker volumes
    rng = np.random.default_rng(8)
    Xs = np.concatenate([synth.fibonacci_sphere(500, sph[b, :3], sph[b, 3])[0] for b in range(2)], axis=1)
    ss = np.array([0, 500, 1000])
    F = rng.normal(size=(3, 1000)).astype(np.float32)
    dV = rng.uniform(0.5, 1.5, 1000).astype(np.float32) * h ** 3
    lin, ang = ot.ot_body_sums(*pts(Xs), dev(F), torch.as_tensor(ss, device="cuda"), xb, -1.0, dV=dev(dV))
    lref, aref = oracle.body_sums(Xs, F.astype(np.float64), ss, sph[:, :3], -1.0, dV=dV.astype(np.float64))
    assert np.allclose(lin.cpu().numpy(), lref, rtol=1e-9, atol=1e-16)
    assert np.allclose(ang.cpu().numpy(), aref, rtol=1e-9, atol=1e-18)
    # deterministic
    lin2, ang2 = ot.ot_body_sums(*pts(Xs), dev(F), torch.as_tensor(ss, device="cuda"), xb, -1.0, dV=dev(dV))
    assert torch.equal(lin, lin2) and torch.equal(ang, ang2)


# ---------------------------------------------------------------------------------------
# Periodic box (Sec. 5.2)
# ---------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def uniform6(ot):
    ko, lo = oracle.octree_build(np.zeros((0, 5)), 6, 6)
    t = ot.ot_octree_build(np.zeros((0, 5)), 6, 6)
    ot.ot_octree_set_periodic(t, True)
    rng = np.random.default_rng(17)
    nc = 64
    P = np.concatenate([rng.uniform(0, 1, (3000, 3)), rng.uniform(0, 1.5 / nc, (1000, 3)),
                        1.0 - rng.uniform(1e-9, 1.5 / nc, (1000, 3))])
    field = np.zeros((ko.size, 4))
    field[:, :3] = rng.normal(size=(ko.size, 3))
    return ko, lo, t, P, field


@pytest.mark.parametrize("kernel", [2, 3])
def test_periodic_delta_interp_and_spread(ot, uniform6, kernel, torch_mod):
    torch = torch_mod
    ko, lo, t, P, field = uniform6
    f32 = field.astype(np.float32)
    u = ot.ot_interpolate(t, kernel, *pts(P.T), dev(f32)).cpu().numpy()
    ref, bad = oracle.interp_delta(ko, lo, 6, kernel, f32.astype(np.float64), *P.T, periodic=True)
    assert bad == 0
    assert rel_err(u, ref) <= TOL32
    rng = np.random.default_rng(3)
    F = rng.normal(size=(3, P.shape[0])).astype(np.float32)
    fref, bad = oracle.spread_delta(ko, lo, 6, kernel, *P.T, F.astype(np.float64), periodic=True)
    assert bad == 0
    for mode in (ot.OT_SORTED, ot.OT_ATOMIC):
        f = torch.zeros((ko.size, 4), dtype=torch.float32, device="cuda")
        ot.ot_spread(t, kernel, mode, *pts(P.T), dev(F), f)
        assert rel_err(f.cpu().numpy()[:, :3], fref[:, :3]) <= TOL32
    assert ot.ot_last_error(t) & ot.OT_DEV_STENCIL == 0


def test_periodic_trilinear(ot, tiny, tiny_fields):
    w, ko, lo, _ = tiny
    t = ot.ot_octree_build(w.spheres, w.lmin, w.lmax)
    ot.ot_octree_set_periodic(t, True)
    rng = np.random.default_rng(21)
    P = np.concatenate([rng.uniform(0, 1, (2000, 3)), rng.uniform(0, 0.02, (500, 3)),
                        1.0 - rng.uniform(1e-9, 0.02, (500, 3))])
    f32 = tiny_fields["sin"].astype(np.float32)
    u = ot.ot_interpolate(t, ot.OT_TRILINEAR, *pts(P.T), dev(f32)).cpu().numpy()
    host = oracle.locate_ub(ko, lo, *P.T)
    ref = oracle.interp_trilinear(ko, lo, f32.astype(np.float64), *P.T, host, periodic=True)
    assert rel_err(u, ref) <= TOL32
    # the batched form keeps the setting
    import torch
    ub = torch.empty((3, P.shape[0]), device="cuda")
    x, y, z = pts(P.T)
    b = ot.ot_batch_create(t, [dict(kernel=ot.OT_TRILINEAR, x=x, y=y, z=z, u=ub)], dev(f32))
    ot.ot_batch_run(b)
    assert rel_err(ub.cpu().numpy(), ref) <= TOL32


def test_field_subtract_mean(ot, tiny, torch_mod):
    w, ko, lo, tree = tiny
    rng = np.random.default_rng(9)
    f = rng.normal(size=(ko.size, 4)).astype(np.float32)
    ref = oracle.field_mean(lo, f.astype(np.float64))
    d = dev(f)
    m = ot.ot_field_subtract_mean(tree, d).cpu().numpy()
    assert np.abs(m - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    out = d.cpu().numpy()
    assert np.abs(out[:, :3] - (f[:, :3] - ref.astype(np.float32))).max() <= 1e-6
    assert np.array_equal(out[:, 3], f[:, 3])
    assert np.abs(oracle.field_mean(lo, out.astype(np.float64))).max() <= 1e-6


@pytest.mark.parametrize("at_rest", [False, True])
def test_marker_force(ot, torch_mod, at_rest):
    """Direct-forcing marker force (Sec. 2.2): F = (U - u) / dt, evaluated as (U - u) * (1/dt) in
    FP32 -- bit for bit the same FP32 operations on the host -- and within FP32 rounding of the
    FP64 quotient."""
    torch = torch_mod
    rng = np.random.default_rng(12)
    n = 5003
    u = rng.normal(size=(3, n)).astype(np.float32)
    U = np.zeros_like(u) if at_rest else rng.normal(size=(3, n)).astype(np.float32)
    dt = 0.37
    F = ot.ot_marker_force(dev(u), dt, U=None if at_rest else dev(U)).cpu().numpy()
    ref32 = (U - u) * (np.float32(1.0) / np.float32(dt))
    assert np.array_equal(F, ref32)
    ref64 = (U.astype(np.float64) - u.astype(np.float64)) / np.float64(np.float32(dt))
    assert np.abs(F - ref64).max() <= 4e-7 * np.abs(ref64).max()
