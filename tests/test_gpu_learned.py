"""The learned index's gain over the method without it, and the launch autotuner (GPU).

Gain: on a tree whose keys cluster (two small refined spheres in a coarse cube), the root
network's routing is compared with a linear root and with no model at all (a binary search of
the whole key array).  The measure is the window a stored key's leaf model leaves to search,
and the halving probes it takes; every form answers bit-identically to the plain search."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ot():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_20565_gb300 as m
    return m


def pts(a):
    import torch
    return [torch.as_tensor(np.ascontiguousarray(a[d], dtype=np.float64)).cuda() for d in range(3)]


@pytest.fixture(scope="module")
def clustered(ot):
    sph = np.array([[0.53, 0.47, 0.51, 0.05, 0.02], [0.2, 0.7, 0.3, 0.03, 0.015]])
    ko, lo = oracle.octree_build(sph, 3, 9)
    rng = np.random.default_rng(5)
    P = np.concatenate([rng.uniform(0, 1, (40000, 3)),
                        sph[0, :3] + rng.normal(0, 0.05, (40000, 3))])
    P = P[np.all((P >= 0) & (P < 1), axis=1)]
    return sph, ko, lo, P


def train_stats(ot, tree, root, n_leaf, n_mid):
    ot.ot_index_train(tree, root=root, n_leaf_models=n_leaf, n_mid_models=n_mid, epochs=4, batch=16384, lr=1e-3,
                      seed=3)
    return ot.ot_index_get_stats(tree, reset=True)


def test_learned_gain_over_linear_root_and_no_model(ot, clustered):
    sph, ko, lo, P = clustered
    tree = ot.ot_octree_build(sph, 3, 9)
    ot.ot_octree_set_map_level(tree, 0)  # no level map: the models alone narrow the search
    n = ko.size
    ref = oracle.locate_ub(ko, lo, *P.T)
    x, y, z = pts(P.T)
    res = {}
    for name, root in (("mlp", ot.OT_ROOT_MLP), ("linear", ot.OT_ROOT_LINEAR)):
        st = train_stats(ot, tree, root, 4096, 0)
        h = ot.ot_locate(tree, x, y, z, search=ot.OT_LEARNED)
        assert np.array_equal(h.cpu().numpy(), ref)
        res[name] = st
    no_model_probes = math.ceil(math.log2(n))
    print("learned-index gain:", {"n": n, "no_model_probes": no_model_probes,
                                  **{f"{k}_{m}": v[m] for k, v in res.items() for m in ("mean_window", "mean_probes")}})
    # the trained network routes the clustered keys far more evenly than a line through the
    # key CDF: smaller windows and fewer probes than the linear root, and both beat searching
    # the whole array
    assert res["mlp"]["mean_window"] < 0.5 * res["linear"]["mean_window"], res
    assert res["mlp"]["mean_probes"] < res["linear"]["mean_probes"] - 1.0, res
    assert res["linear"]["mean_probes"] < no_model_probes, res
    assert res["mlp"]["mean_probes"] <= no_model_probes - 5, res


def test_three_stage_index_narrows_windows_further(ot, clustered):
    sph, ko, lo, P = clustered
    tree = ot.ot_octree_build(sph, 3, 9)
    two = train_stats(ot, tree, ot.OT_ROOT_MLP, 4096, 0)
    three = train_stats(ot, tree, ot.OT_ROOT_MLP, 1 << 16, 1024)
    h = ot.ot_locate(tree, *pts(P.T), search=ot.OT_LEARNED)
    assert np.array_equal(h.cpu().numpy(), oracle.locate_ub(ko, lo, *P.T))
    print("two-stage vs three-stage:", two["mean_probes"], three["mean_probes"])
    assert three["mean_probes"] < two["mean_probes"], (two, three)


def test_autotune_picks_a_valid_shape_and_keeps_results(ot):
    import torch
    from paper_2605_20565_gb300 import synth
    w = synth.tiny()
    tree = ot.ot_octree_build(w.spheres, w.lmin, w.lmax)
    cen = ot.ot_octree_centres(tree).cpu().numpy()
    field = torch.as_tensor(synth.sin_field(cen.T).astype(np.float32)).cuda()
    mx, my, mz = pts(w.markers)
    px, py, pz = pts(w.particles)
    um = torch.empty((3, w.markers.shape[1]), device="cuda")
    up = torch.empty((3, w.particles.shape[1]), device="cuda")
    groups = [dict(kernel=ot.OT_PESKIN4, x=mx, y=my, z=mz, u=um), dict(kernel=ot.OT_TRILINEAR, x=px, y=py, z=pz, u=up)]
    ref_m = ot.ot_interpolate(tree, ot.OT_PESKIN4, mx, my, mz, field)
    ref_p = ot.ot_interpolate(tree, ot.OT_TRILINEAR, px, py, pz, field)
    r = ot.ot_batch_autotune(tree, groups, field, search=ot.OT_BINARY, tune_map_level=True, reps=1)
    assert r["tried"] == 32  # lmax 5: one level-map level, 32 launch shapes (16 with the points ordered)
    assert r["map_level"] == 5 and r["ms"] > 0
    assert r["launch"]["block"] in (128, 256) and r["launch"]["tile"] in (1, 2, 4, 8)
    assert r["launch"]["order_level"] in (0, 8)
    b = ot.ot_batch_create(tree, groups, field, search=ot.OT_BINARY, launch=r["launch"])
    ot.ot_batch_run(b)
    torch.cuda.synchronize()
    assert torch.equal(um, ref_m) and torch.equal(up, ref_p)


def test_warm_start_keeps_the_network_and_stays_exact(ot, clustered):
    sph, ko, lo, P = clustered
    tree = ot.ot_octree_build(sph, 3, 9)
    ot.ot_index_train(tree, root=ot.OT_ROOT_MLP, n_leaf_models=4096, epochs=2, batch=16384, seed=5)
    p0 = ot.ot_index_get_root_params(tree)
    t2 = ot.ot_octree_build(sph, 3, 9)
    ot.ot_index_train(t2, root=ot.OT_ROOT_MLP, n_leaf_models=4096, epochs=0, init=p0)
    assert np.array_equal(ot.ot_index_get_root_params(t2), p0)  # no steps: the starting network
    ot.ot_index_train(t2, root=ot.OT_ROOT_MLP, n_leaf_models=4096, steps=16, init=p0, lr=1e-4)
    h = ot.ot_locate(t2, *pts(P.T), search=ot.OT_LEARNED)
    assert np.array_equal(h.cpu().numpy(), oracle.locate_ub(ko, lo, *P.T))
