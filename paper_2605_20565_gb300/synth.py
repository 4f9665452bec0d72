"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the only code that both the CUDA path and the CPU oracle are fed from.  It
holds no arithmetic of the method itself (no search, no interpolation, no delta kernels, no
spreading): it draws sphere lists, marker and particle positions, forces and velocity fields.
One helper, marker_morton_order, computes level-10 Morton keys of the markers, but only to
choose the order in which the markers are stored; that permutation is applied to the input
arrays before either side sees them, so both sides receive the same reordered inputs.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), used as a
counter-based generator: value i of stream s under seed S is splitmix64_mix(base(S, s) +
(i + 1) * GAMMA).  Uniform doubles take the top 53 bits; normals use Box-Muller.  The
recipe is pure integer arithmetic and gives the same bits on x86-64 and aarch64.

Workload shapes (stand-ins for the paper's runs; no dataset is involved):
  * one bubble with an l_max shell around it (the rising-bubble run of Sec. 5.1);
  * many bubbles of disparate size plus many point particles (the HIT run of Sec. 5.2);
  * 10^7 uniform points (the host-search benchmark of Sec. 3.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_base(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([(seed * 1_000_003 + stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix(s * _GAMMA + _GAMMA)[0]


def bits(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n raw 64-bit values of (seed, stream), starting at counter ``offset``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(_stream_base(seed, stream) + i * _GAMMA)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1)."""
    return (bits(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


# ---------------------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------------------

def fibonacci_sphere(n: int, centre, radius: float):
    """n points on a sphere by the Fibonacci lattice (z_i = 1 - (2i+1)/n, longitude
    i * pi * (3 - sqrt 5)); returns positions (3, n) and outward unit normals (3, n)."""
    i = np.arange(n, dtype=np.float64)
    zc = 1.0 - (2.0 * i + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - zc * zc))
    lon = i * math.pi * (3.0 - math.sqrt(5.0))
    nrm = np.stack([rho * np.cos(lon), rho * np.sin(lon), zc])
    pos = np.asarray(centre, np.float64).reshape(3, 1) + radius * nrm
    return pos, nrm


def largest_remainder(total: int, weights) -> np.ndarray:
    """Split ``total`` into integers proportional to ``weights`` (largest-remainder rule)."""
    w = np.asarray(weights, np.float64)
    q = total * w / w.sum()
    base = np.floor(q).astype(np.int64)
    rest = total - int(base.sum())
    order = np.argsort(-(q - base), kind="stable")
    base[order[:rest]] += 1
    return base


def place_bubbles(seed: int, n: int, dmin: float, dmax: float, wall: str = "d", max_tries: int = 200000,
                  extra_margin: float = 0.0):
    """n non-overlapping bubbles, diameters log-uniform in [dmin, dmax], centres at least one
    diameter (plus ``extra_margin``) from every wall (``wall='d'``) and |c_i - c_j| >= r_i + r_j.
    Rejection sampling on one counter stream; returns centres (n, 3) and diameters (n,)."""
    cs, ds = [], []
    t = 0
    while len(cs) < n:
        if t >= max_tries:
            raise RuntimeError("bubble placement did not converge")
        u = uniform(seed, 10, 4, offset=4 * t)
        t += 1
        d = dmin * (dmax / dmin) ** u[0]
        m = (d + extra_margin) if wall == "d" else 0.0
        c = m + (1.0 - 2.0 * m) * u[1:4]
        ok = all(np.linalg.norm(c - c2) >= 0.5 * (d + d2) for c2, d2 in zip(cs, ds))
        if ok:
            cs.append(c)
            ds.append(d)
    return np.array(cs), np.array(ds)


# ---------------------------------------------------------------------------------------
# Velocity fields
# ---------------------------------------------------------------------------------------

@dataclass
class FourierModes:
    """u(x) = sum_m A_m cos(2 pi n_m . x + phase_m), n_m integer with 1 <= |n_m| <= nmax,
    A_m orthogonal to n_m (so div u = 0), |A_m| = |n_m|^(-5/3) (amplitude, read literally)."""
    n: np.ndarray      # (M, 3) integer wave vectors
    amp: np.ndarray    # (M, 3)
    phase: np.ndarray  # (M,)


def fourier_modes(seed: int, n_modes: int = 32, nmax: int = 8) -> FourierModes:
    ns, t = [], 0
    while len(ns) < n_modes:
        u = uniform(seed, 20, 3, offset=3 * t)
        t += 1
        v = np.floor(u * (2 * nmax + 1)).astype(np.int64) - nmax
        r = math.sqrt(float((v * v).sum()))
        if 1.0 <= r <= nmax:
            ns.append(v)
    ns = np.array(ns)
    g = normal(seed, 21, 3 * n_modes).reshape(n_modes, 3)
    nn = ns / np.linalg.norm(ns, axis=1, keepdims=True)
    a = g - (g * nn).sum(1, keepdims=True) * nn
    a = a / np.linalg.norm(a, axis=1, keepdims=True)
    a = a * (np.linalg.norm(ns, axis=1, keepdims=True) ** (-5.0 / 3.0))
    ph = 2.0 * math.pi * uniform(seed, 22, n_modes)
    return FourierModes(ns.astype(np.float64), a, ph)


def fourier_field(modes: FourierModes, centres, chunk: int = 1 << 20):
    """Evaluate the modes at points ``centres`` ((N, 3) numpy float64, or a torch tensor on
    any device).  Returns (N, 4) float64 with component 3 zero, same library as input."""
    try:
        import torch  # noqa: F401
        is_torch = not isinstance(centres, np.ndarray)
    except ImportError:  # pragma: no cover
        is_torch = False
    if is_torch:
        # On a GPU: the phase in turns in FP64 (exact integer wave vectors), reduced to
        # [-1/2, 1/2), then the cosine in FP32 (GB300's FP64 rate makes an FP64 cosine of 10^9
        # arguments the slow part); the mode sum in FP64.  Differs from the FP64 evaluation by
        # ~1e-7 of max|u|.
        import torch
        dev = centres.device
        kn = torch.as_tensor(modes.n, dtype=torch.float64, device=dev)
        am = torch.as_tensor(modes.amp, dtype=torch.float64, device=dev)
        ph = torch.as_tensor(modes.phase / (2.0 * math.pi), dtype=torch.float64, device=dev)
        out = torch.zeros((centres.shape[0], 4), dtype=torch.float64, device=dev)
        big = max(chunk, 1 << 22)
        for s in range(0, centres.shape[0], big):
            c = centres[s:s + big].to(torch.float64)
            turns = c @ kn.T + ph
            turns = turns - torch.floor(turns + 0.5)
            cs = torch.cos((2.0 * math.pi) * turns.to(torch.float32)).to(torch.float64)
            out[s:s + big, :3] = cs @ am
        return out
    c = np.asarray(centres, np.float64)
    out = np.zeros((c.shape[0], 4), np.float64)
    for s in range(0, c.shape[0], chunk):
        arg = 2.0 * math.pi * (c[s:s + chunk] @ modes.n.T) + modes.phase
        out[s:s + chunk, :3] = np.cos(arg) @ modes.amp
    return out


def sin_field(centres):
    """u = (sin 2 pi y, sin 2 pi z, sin 2 pi x)."""
    c = np.asarray(centres, np.float64)
    out = np.zeros((c.shape[0], 4))
    out[:, 0] = np.sin(2 * np.pi * c[:, 1])
    out[:, 1] = np.sin(2 * np.pi * c[:, 2])
    out[:, 2] = np.sin(2 * np.pi * c[:, 0])
    return out


LINEAR_COEF = np.array([[1.0, 2.0, -1.0, 0.5],
                        [-1.0, 1.0, 3.0, -2.0],
                        [0.5, -1.0, 0.25, 1.0]])  # rows: u_d = a + b x + c y + e z


def linear_field(points):
    """The linear test field u_d = LINEAR_COEF[d] . (1, x, y, z); (N, 4), component 3 zero."""
    p = np.asarray(points, np.float64).reshape(-1, 3)
    out = np.zeros((p.shape[0], 4))
    out[:, :3] = LINEAR_COEF[:, 0] + p @ LINEAR_COEF[:, 1:].T
    return out


# ---------------------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    seed: int
    lmin: int
    lmax: int
    spheres: np.ndarray            # (S, 5): cx, cy, cz, r, w
    markers: np.ndarray            # (3, N_m) positions
    forces: np.ndarray             # (3, N_m) marker forces F_k
    marker_group: np.ndarray       # (N_m,) bubble id of each marker
    particles: np.ndarray          # (3, N_p) positions
    modes: FourierModes | None = None
    extra: dict = field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return self.markers.shape[1] + self.particles.shape[1]


def _uniform_points(seed: int, stream: int, n: int) -> np.ndarray:
    return uniform(seed, stream, 3 * n).reshape(n, 3).T.copy()


def _clustered_points(seed: int, stream: int, n: int, centre, sigma: float) -> np.ndarray:
    """n points from N(centre, sigma^2 I), each redrawn until it lies in [0,1)^3."""
    out = np.empty((n, 3))
    todo = np.arange(n)
    attempt = 0
    c = np.asarray(centre, np.float64)
    while todo.size:
        g = normal(seed, stream + 1000 * attempt, 3 * n).reshape(n, 3)[todo]
        p = c + sigma * g
        ok = np.all((p >= 0.0) & (p < 1.0), axis=1)
        out[todo[ok]] = p[ok]
        todo = todo[~ok]
        attempt += 1
    return out.T.copy()


def _markers_on(centres, diams, counts, seed):
    pos, nrm, grp = [], [], []
    for b, (c, d, m) in enumerate(zip(centres, diams, counts)):
        if m == 0:
            continue
        p, nv = fibonacci_sphere(int(m), c, 0.5 * d)
        pos.append(p)
        nrm.append(nv)
        grp.append(np.full(int(m), b, np.int32))
    return np.concatenate(pos, 1), np.concatenate(nrm, 1), np.concatenate(grp)


def marker_morton_order(markers: np.ndarray, groups: np.ndarray, level: int = 10) -> np.ndarray:
    """The permutation that stores markers bubble by bubble, each bubble's in Morton order of
    the level-``level`` cells holding them (consecutive markers are then neighbours on the
    surface: a warp's markers share parent blocks and stencil cells)."""
    if markers.shape[1] == 0:
        return np.arange(0)
    q = np.floor(np.clip(markers, 0.0, np.nextafter(1.0, 0.0)) * float(1 << level)).astype(np.uint64)
    key = np.zeros(q.shape[1], np.uint64)
    for b in range(level):
        for d in range(3):
            key |= ((q[d] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + d)
    return np.lexsort((key, groups))


def order_markers(w: Workload) -> np.ndarray:
    """Stores the workload's markers (positions, forces, groups) in marker_morton_order; returns
    the permutation (stored marker i is input marker perm[i])."""
    perm = marker_morton_order(w.markers, w.marker_group)
    w.markers = np.ascontiguousarray(w.markers[:, perm])
    w.forces = np.ascontiguousarray(w.forces[:, perm])
    w.marker_group = np.ascontiguousarray(w.marker_group[perm])
    return perm


def internal_markers(centres, diameters, h: float):
    """Lagrangian points inside each body on a cubic lattice of spacing h centred on the body
    (the internal markers of Sec. 2.3, spacing the finest cell): the points c + h (i, j, k)
    with |h (i, j, k)| < r - h/2.  Returns positions (3, n) grouped by body and the offsets
    start (nb + 1,) of each body's markers."""
    centres = np.asarray(centres, np.float64).reshape(-1, 3)
    diameters = np.asarray(diameters, np.float64).reshape(-1)
    pts, start = [], [0]
    for c, d in zip(centres, diameters):
        r = 0.5 * d
        m = int(np.floor(r / h))
        g = np.arange(-m, m + 1, dtype=np.float64) * h
        gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
        off = np.stack([gx.ravel(), gy.ravel(), gz.ravel()])
        keep = (off ** 2).sum(0) < (r - 0.5 * h) ** 2
        pts.append(c[:, None] + off[:, keep])
        start.append(start[-1] + int(keep.sum()))
    X = np.concatenate(pts, axis=1) if pts else np.zeros((3, 0))
    return np.ascontiguousarray(X), np.asarray(start, np.int64)


def tiny(seed: int = 0) -> Workload:
    """Levels 3-5 refined to 5 within 0.1 of the sphere c = (.5,.5,.5), r = 0.2; 1,000
    Fibonacci markers with F = outward unit normal; 10,000 uniform particles."""
    c = np.array([0.5, 0.5, 0.5])
    sph = np.array([[0.5, 0.5, 0.5, 0.2, 0.1]])
    pos, nrm = fibonacci_sphere(1000, c, 0.2)
    return Workload("tiny_fp64_l3-5", seed, 3, 5, sph, pos, nrm.copy(), np.zeros(1000, np.int32),
                    _uniform_points(seed, 1, 10000))


def single_bubble(seed: int = 1, n_markers: int = 50_000, n_particles: int = 10_000_000) -> Workload:
    """Levels 5-9, level 9 within two diameters (w = 0.2) of a d = 0.1 bubble at a centre
    uniform in [0.2, 0.8]^3; markers on the bubble; half the particles uniform, half
    N(centre, 0.05^2 I) inside the cube."""
    c = 0.2 + 0.6 * uniform(seed, 2, 3)
    d = 0.1
    sph = np.array([[c[0], c[1], c[2], 0.5 * d, 2.0 * d]])
    pos, nrm = fibonacci_sphere(n_markers, c, 0.5 * d)
    half = n_particles // 2
    parts = np.concatenate([_uniform_points(seed, 3, half),
                            _clustered_points(seed, 4, n_particles - half, c, 0.05)], 1)
    return Workload("single_bubble_l5-9", seed, 5, 9, sph, pos, nrm.copy(), np.zeros(n_markers, np.int32),
                    parts, fourier_modes(seed))


# Shell half-width as a multiple of the bubble diameter, chosen so that the leaf counts of
# the many-bubble workloads land near the stated sizes: ~30M leaves for 64 bubbles at level
# 10 (the literal two-diameter shell gives about 10^8) and ~80M for 256 bubbles at level 11.
MANY_BUBBLE_SHELL = 0.25
TRACKING_SHELL = 0.06


def many_bubbles(seed: int = 2, n_markers: int = 2_000_000, n_particles: int = 50_000_000,
                 shell: float = MANY_BUBBLE_SHELL, lmin: int = 4, lmax: int = 10) -> Workload:
    """64 non-overlapping bubbles, d log-uniform in [0.02, 0.1], levels 4-10 with the finest
    level in each bubble's shell; markers split in proportion to d^2; uniform particles."""
    cs, ds = place_bubbles(seed, 64, 0.02, 0.1)
    sph = np.column_stack([cs, 0.5 * ds, shell * ds])
    counts = largest_remainder(n_markers, ds ** 2)
    pos, nrm, grp = _markers_on(cs, ds, counts, seed)
    return Workload(f"many_bubbles_l{lmin}-{lmax}", seed, lmin, lmax, sph, pos, nrm, grp,
                    _uniform_points(seed, 3, n_particles), fourier_modes(seed),
                    extra={"centres": cs, "diameters": ds})


def learned_index(seed: int = 3, n_particles: int = 100_000_000, n_markers: int = 0) -> Workload:
    """The many-bubble octree (same sphere list and seed as ``many_bubbles``); 70 % uniform
    particles and 30 % near bubble surfaces (bubble chosen in proportion to d^2, uniform
    direction, radial offset N(0, (0.1 r)^2))."""
    base = many_bubbles(seed=2, n_markers=max(n_markers, 64), n_particles=0)
    cs, ds = base.extra["centres"], base.extra["diameters"]
    n_u = int(round(0.7 * n_particles))
    n_s = n_particles - n_u
    uni = _uniform_points(seed, 3, n_u)
    cdf = np.cumsum(ds ** 2) / np.sum(ds ** 2)
    pick = np.searchsorted(cdf, uniform(seed, 5, n_s), side="right")
    pick = np.minimum(pick, len(ds) - 1)
    g = normal(seed, 6, 3 * n_s).reshape(n_s, 3)
    g = g / np.linalg.norm(g, axis=1, keepdims=True)
    rad = 0.5 * ds[pick] * (1.0 + 0.1 * normal(seed, 7, n_s))
    p = cs[pick] + g * rad[:, None]
    p = np.clip(p, 0.0, np.nextafter(1.0, 0.0))
    parts = np.concatenate([uni, p.T], 1)
    mk = base.markers[:, :n_markers] if n_markers else np.zeros((3, 0))
    fk = base.forces[:, :n_markers] if n_markers else np.zeros((3, 0))
    return Workload("learned_index_l4-10", seed, base.lmin, base.lmax, base.spheres, mk, fk,
                    np.zeros(mk.shape[1], np.int32), parts, base.modes, extra=base.extra)


def tracking(seed: int = 4, n_particles: int = 200_000_000, shell: float = TRACKING_SHELL,
             lmin: int = 4, lmax: int = 11, n_bubbles: int = 256) -> Workload:
    """256 bubbles, d log-uniform in [0.01, 0.08], levels 4-11, shell max(0.06 d, 4 h); markers
    per bubble round(pi (d/h)^2) at h = 2^-lmax; uniform particles; bubble velocities in extra."""
    h = 2.0 ** -lmax
    cs, ds = place_bubbles(seed, n_bubbles, 0.01, 0.08, extra_margin=4.0 * h)  # stencils stay inside
    # at least 4 finest cells: the 4-point stencil of every marker (reach ~2.6 h) stays on the
    # finest level while the bubbles move between re-adaptations
    sph = np.column_stack([cs, 0.5 * ds, np.maximum(shell * ds, 4.0 * h)])
    counts = np.round(np.pi * (ds / h) ** 2).astype(np.int64)
    pos, nrm, grp = _markers_on(cs, ds, counts, seed)
    vel = 0.05 * normal(seed, 8, 3 * n_bubbles).reshape(n_bubbles, 3)
    return Workload(f"tracking_l{lmin}-{lmax}", seed, lmin, lmax, sph, pos, nrm, grp,
                    _uniform_points(seed, 3, n_particles), fourier_modes(seed),
                    extra={"centres": cs, "diameters": ds, "velocities": vel})
