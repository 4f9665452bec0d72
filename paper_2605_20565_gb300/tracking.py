"""Time-stepped tracking of point particles among moving bubbles (Sec. 2.3.2 particle
update; Sec. 2.4 re-adaptation; Algorithm 2's post-refinement re-location on one GPU).

Every step, through the C ABI:
  1. one batched launch locates and interpolates every IBM marker (Peskin-4) and every point
     particle (trilinear) -- ``ot_batch_run``;
  2. the particles advance by AB2 with Schiller-Naumann drag (``ot_advect_ab2``, periodic
     wrap into the unit cube);
  3. the marker forces are spread back to the cells by the deterministic sorted reduction
     (``ot_spread``);
  4. the bubbles translate at constant velocities carrying their markers.
Every ``rebuild_every`` steps the octree is rebuilt around the moved bubbles
(``ot_octree_build``) with its level-mate table (``ot_octree_build_mates``), the learned
index is retrained on the device for the learned form (``ot_index_train``), the velocity
field is re-sampled at the new leaf centres, the particles are re-stored in Morton
order of their cells (``ot_points_morton_order``; ``ids`` keeps each one's original index),
and the batch graph is re-captured: the single-GPU form of re-locating every point after a
mesh change.

The time step keeps particle motion below one finest cell per step: dt = h_lmax / max|u|.
"""
from __future__ import annotations

import time

import numpy as np

from . import synth


class Tracker:
    def __init__(self, w: synth.Workload, search: int = 1, rebuild_every: int = 10, tau_steps: float = 10.0,
                 re_coef: float = 0.0, n_leaf_models: int = 1 << 18, n_mid_models: int = 4096, device=None,
                 sort_points: bool = True, mates: bool = True, map_level: int | None = None,
                 launch: dict | None = None, autotune: bool = True, dt: float | None = None):
        import torch
        from . import OT_PESKIN4, OT_SORTED, OT_TRILINEAR
        self.torch = torch
        self.w = w
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.search = search
        self.rebuild_every = rebuild_every
        self.re_coef = re_coef
        self.n_leaf_models = n_leaf_models
        self.n_mid_models = n_mid_models
        self.centres0 = np.asarray(w.extra["centres"], np.float64)
        self.vel = np.asarray(w.extra["velocities"], np.float64)
        self.radii = 0.5 * np.asarray(w.extra["diameters"], np.float64)
        self.shells = w.spheres[:, 4].copy()
        self.t = 0.0
        self.step_no = 0
        T = torch
        dev = self.dev
        self.x = T.as_tensor(np.ascontiguousarray(w.particles), device=dev)            # (3, n) FP64
        n = self.x.shape[1]
        self.sort_points = sort_points
        self.mates = mates  # level-mate table built with every octree
        self.map_level = map_level  # level-map level of every octree (None: the library's default)
        self.launch = launch  # launch shape of the batch (None: the library's default)
        self.ids = T.arange(n, device=dev)  # original index of each stored particle
        self.v = T.zeros((3, n), dtype=T.float32, device=dev)
        self.a_prev = T.zeros_like(self.v)
        self.v_prev = T.zeros_like(self.v)
        self.u = T.empty_like(self.v)
        # markers: offsets from their bubble centre (moved rigidly), forces = outward normals.
        # Stored bubble by bubble in Morton order of their initial positions (a rigid motion
        # keeps neighbours neighbours), so a warp's markers share parent blocks; m_ids maps
        # each stored marker to its input index.
        m_ids = np.arange(w.markers.shape[1])
        if sort_points and w.markers.shape[1] > 0:
            m_ids = synth.marker_morton_order(w.markers, w.marker_group)
        self.m_ids = T.as_tensor(m_ids, device=dev)
        self.m_grp = T.as_tensor(w.marker_group[m_ids].astype(np.int64), device=dev)
        self.m_off = T.as_tensor(np.ascontiguousarray((w.markers - self.centres0[w.marker_group].T)[:, m_ids]),
                                 device=dev)
        self.mx = T.empty((3, w.markers.shape[1]), dtype=T.float64, device=dev)
        self.F = T.as_tensor(np.ascontiguousarray(w.forces[:, m_ids], dtype=np.float32), device=dev)
        self.um = T.empty((3, w.markers.shape[1]), dtype=T.float32, device=dev)
        self._place_markers()
        self.h = 2.0 ** -w.lmax
        self.kinds = (OT_PESKIN4, OT_SORTED, OT_TRILINEAR)
        self.ws = T.empty(1, dtype=T.uint8, device=dev)  # sized at the first rebuild
        self.timings = {"rebuild_s": 0.0, "rebuilds": 0}
        self._rebuild()
        if autotune and launch is None:
            # the launch shape for this point order (the trilinear launch wants more resident
            # warps for Morton-ordered particles than for random ones), tuned once on the
            # first octree and kept for the later ones
            import paper_2605_20565_gb300 as ot
            K_P4, _, K_TRI = self.kinds
            groups = [dict(kernel=K_P4, x=self.mx[0], y=self.mx[1], z=self.mx[2], u=self.um),
                      dict(kernel=K_TRI, x=self.x[0], y=self.x[1], z=self.x[2], u=self.u)]
            r = ot.ot_batch_autotune(self.tree, groups, self.field, search=self.search, tune_map_level=False,
                                     reps=2)
            self.launch = r["launch"]
            self.tuned = r
            self.batch = ot.ot_batch_create(self.tree, groups, self.field, search=self.search, launch=self.launch)
        if dt is None:
            umax = float(self.field[:, :3].abs().max())
            dt = self.h / max(umax, 1e-12)
        self.dt = dt
        self.tau = tau_steps * self.dt

    def spheres_now(self) -> np.ndarray:
        c = self.centres0 + self.vel * self.t
        return np.column_stack([c, self.radii, self.shells])

    def _place_markers(self):
        c = self.torch.as_tensor(self.centres0 + self.vel * self.t, device=self.dev)  # (B, 3)
        self.mx.copy_(c[self.m_grp].T + self.m_off)

    def markers_at(self, t: float) -> np.ndarray:
        """The markers' positions (3, n) at time t in the input order, computed on the host from
        the input positions and the bubble velocities (rigid translation)."""
        w = self.w
        return w.markers + (self.vel[w.marker_group] * t).T

    def _reorder(self):
        """Store the particles in Morton order of their cells (neighbouring particles share host
        leaves and level-mates in a warp); every per-particle array follows."""
        import paper_2605_20565_gb300 as ot
        perm = ot.ot_points_morton_order(self.x[0], self.x[1], self.x[2]).long()
        for name in ("x", "v", "a_prev", "v_prev", "u", "ids"):
            a = getattr(self, name)
            setattr(self, name, a.index_select(a.dim() - 1, perm).contiguous())

    def _rebuild(self):
        import paper_2605_20565_gb300 as ot
        T = self.torch
        t0 = time.time()
        w = self.w
        parts = self.timings.setdefault("rebuild_parts_s", {})

        def mark(name, t_prev):
            T.cuda.synchronize()
            now = time.time()
            parts[name] = parts.get(name, 0.0) + now - t_prev
            return now

        t = t0
        if self.sort_points:
            self._reorder()
            t = mark("reorder", t)
        prev = (ot.ot_index_get_root_params(self.tree)
                if self.search == ot.OT_LEARNED and getattr(self, "tree", None) is not None else None)
        # the spheres, time and step of this octree (for checks against an independent build)
        self.tree_spheres, self.tree_time, self.tree_step = self.spheres_now(), self.t, self.step_no
        self.tree = ot.ot_octree_build(self.tree_spheres, w.lmin, w.lmax)
        if self.map_level is not None:
            ot.ot_octree_set_map_level(self.tree, self.map_level)
        t = mark("octree_build", t)
        if self.mates:
            # one table buffer for every octree (grown with 10% headroom when a tree outgrows it):
            # no allocation and release of ~256 bytes per leaf at every re-adaptation
            need = ot.ot_octree_mates_bytes(self.tree)
            buf = getattr(self, "_mates_buf", None)
            if buf is None or buf.numel() < need:
                self._mates_buf = buf = None
                self._mates_buf = T.empty(need + need // 10, dtype=T.uint8, device=self.dev)
            ot.ot_octree_build_mates_in(self.tree, self._mates_buf)
            t = mark("level_mate_table", t)
        # the learned form's index (the plain form needs none): the first trains from the spline
        # initialisation; later ones fine-tune the previous network (the bubbles moved by a few
        # cells): a warm start with few steps
        if self.search == ot.OT_LEARNED:
            ot.ot_index_train(self.tree, root=ot.OT_ROOT_MLP, n_leaf_models=self.n_leaf_models,
                              n_mid_models=self.n_mid_models, epochs=2, batch=65536, lr=1e-3, seed=self.step_no,
                              steps=0 if prev is None else 64, init=prev)
            t = mark("index_train", t)
        n_leaves = ot.ot_octree_info(self.tree)[0]
        self.field = ot.ot_field_fourier(self.tree, w.modes.n, w.modes.amp, w.modes.phase)
        self.f = T.zeros((n_leaves, 4), dtype=T.float32, device=self.dev)
        t = mark("field", t)
        mx, my, mz = self.mx[0], self.mx[1], self.mx[2]
        px, py, pz = self.x[0], self.x[1], self.x[2]
        K_P4, _, K_TRI = self.kinds
        self.batch = ot.ot_batch_create(self.tree, [dict(kernel=K_P4, x=mx, y=my, z=mz, u=self.um),
                                                    dict(kernel=K_TRI, x=px, y=py, z=pz, u=self.u)],
                                        self.field, search=self.search, launch=self.launch)
        need = ot.ot_spread_workspace_size(self.tree, K_P4, self.mx.shape[1])
        if self.ws.numel() < need:
            self.ws = T.empty(need, dtype=T.uint8, device=self.dev)
        mark("batch", t)
        self.timings["rebuild_s"] += time.time() - t0
        self.timings["rebuilds"] += 1

    def step(self, events=None):
        """One coupled step; returns the number of points located and interpolated.  events: an
        optional list of 5 CUDA events recorded between the parts (batch, advect, spread,
        markers)."""
        import paper_2605_20565_gb300 as ot
        K_P4, K_SORTED, _ = self.kinds
        rec = (lambda k: events[k].record()) if events else (lambda k: None)
        rec(0)
        ot.ot_batch_run(self.batch)
        rec(1)
        ot.ot_advect_ab2(self.x, self.v, self.a_prev, self.v_prev, self.u, self.tau, self.re_coef, self.dt,
                         first=self.step_no == 0, periodic=True)
        rec(2)
        self.f.zero_()
        ot.ot_spread(self.tree, K_P4, K_SORTED, self.mx[0], self.mx[1], self.mx[2], self.F, self.f, workspace=self.ws)
        rec(3)
        self.step_no += 1
        self.t += self.dt
        self._place_markers()
        rec(4)
        if self.step_no % self.rebuild_every == 0:
            self._rebuild()
        return self.x.shape[1] + self.mx.shape[1]


def scaled_tracking(n_particles: int, n_bubbles: int = 256, lmax: int = 11, seed: int = 4) -> synth.Workload:
    """The tracking workload with a chosen particle count (the full size is 200M)."""
    return synth.tracking(seed=seed, n_particles=n_particles, lmax=lmax, n_bubbles=n_bubbles)


__all__ = ["Tracker", "scaled_tracking"]
