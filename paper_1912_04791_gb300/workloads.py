"""Seeded synthetic inputs for the A-DOT workloads.

This module only lays out initial data and random states (shapes, sizes and
value ranges of the paper's tests and of the benchmark configurations). It
holds none of the scheme's arithmetic, and both the CUDA path and the oracle
take its arrays as plain inputs.

Conventions: a state is three float64 arrays (h, q, z) on uniform cells of
[x_min, x_max], cell centres x_i = x_min + (i + 1/2) dx. q = h u.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

G = 9.81
XI_P04 = 1.0 / (1.0 - 0.4)  # porosity p = 0.4

# boundary kinds (same meaning on both sides of the boundary; values below)
BC_TRANSMISSIVE, BC_PERIODIC, BC_INFLOW_Q, BC_OUTFLOW_H, BC_INFLOW_QZ, BC_INFLOW_QS, \
    BC_OUTFLOW_HS = range(7)


@dataclass
class Problem:
    name: str
    n: int
    x_min: float
    x_max: float
    cfl: float
    t_end: float
    Ag: float
    xi: float
    h: np.ndarray
    q: np.ndarray
    z: np.ndarray
    bc_left: int = BC_TRANSMISSIVE
    bc_right: int = BC_TRANSMISSIVE
    bcl: tuple = (0.0, 0.0, 0.0)
    bcr: tuple = (0.0, 0.0, 0.0)
    g: float = G
    extra: dict = field(default_factory=dict)

    @property
    def dx(self) -> float:
        return (self.x_max - self.x_min) / self.n


def cell_centres(n: int, x_min: float, x_max: float) -> np.ndarray:
    dx = (x_max - x_min) / n
    return x_min + (np.arange(n, dtype=np.float64) + 0.5) * dx


def riemann(n: int, x_min: float, x_max: float, x0: float, WL, WR) -> tuple:
    """Piecewise-constant data: cells with centre <= x0 take WL=(h,q,z), others WR."""
    x = cell_centres(n, x_min, x_max)
    left = x <= x0
    out = []
    for k in range(3):
        out.append(np.where(left, WL[k], WR[k]).astype(np.float64))
    return tuple(out)


def movable_bed_riemann(n: int = 200) -> Problem:
    """Movable-bed Riemann problem on [0, 10] m, discontinuity at 5 m:
    left h=2.0, u=0.25, z=0; right h=1.0, u=0.2, z=0.5; Grass A_g=0.01,
    p=0.4, CFL 0.9, t_end 1 s, transmissive ends."""
    h, q, z = riemann(n, 0.0, 10.0, 5.0, (2.0, 0.5, 0.0), (1.0, 0.2, 0.5))
    return Problem("movable_bed_riemann", n, 0.0, 10.0, 0.9, 1.0, 0.01, XI_P04, h, q, z)


def smooth_periodic(n: int) -> Problem:
    """Smooth periodic problem on [0, 1] m: h = 1 + 0.1 sin 2 pi x,
    u = 0.3 + 0.05 cos 2 pi x, z = 0.1 sin 2 pi x at cell centres; Grass
    A_g = 0.005, p = 0.4, CFL 0.8, t_end 0.5 s."""
    x = cell_centres(n, 0.0, 1.0)
    h = 1.0 + 0.1 * np.sin(2 * np.pi * x)
    u = 0.3 + 0.05 * np.cos(2 * np.pi * x)
    z = 0.1 * np.sin(2 * np.pi * x)
    return Problem("smooth_periodic", n, 0.0, 1.0, 0.8, 0.5, 0.005, XI_P04, h, h * u, z,
                   BC_PERIODIC, BC_PERIODIC)


def gaussian_bump(n: int, Ag: float = 0.001) -> Problem:
    """Flow over a Gaussian bump z = 0.2 exp(-(x-5)^2) on [0, 10] m with
    h + z = 0.4, q = 0.6; inflow q = 0.6, outflow h = 0.33."""
    x = cell_centres(n, 0.0, 10.0)
    z = 0.2 * np.exp(-(x - 5.0) ** 2)
    h = 0.4 - z
    q = np.full(n, 0.6)
    return Problem("gaussian_bump", n, 0.0, 10.0, 0.9, 10.0, Ag, XI_P04, h, q, z,
                   BC_INFLOW_Q, BC_OUTFLOW_H, (0.6, 0.0, 0.0), (0.33, 0.0, 0.0))


def gaussian_bump_prolonged(h_coarse, q_coarse, n: int, Ag: float = 0.001) -> Problem:
    """The bump flow at n cells from a coarser state of the same problem (e.g. a
    fixed-bed spin-up on a coarse grid): the free surface h + z and q linearly
    interpolated to the fine cell centres (held constant beyond the outer
    centres), the bed z = 0.2 exp(-(x-5)^2) taken at the fine centres, h = (h +
    z) - z. Same boundary data as gaussian_bump."""
    m = len(h_coarse)
    xc = cell_centres(m, 0.0, 10.0)
    zc = 0.2 * np.exp(-(xc - 5.0) ** 2)
    x = cell_centres(n, 0.0, 10.0)
    z = 0.2 * np.exp(-(x - 5.0) ** 2)
    eta = np.interp(x, xc, np.asarray(h_coarse) + zc)
    q = np.interp(x, xc, np.asarray(q_coarse))
    return Problem("gaussian_bump", n, 0.0, 10.0, 0.9, 10.0, Ag, XI_P04, eta - z, q, z,
                   BC_INFLOW_Q, BC_OUTFLOW_H, (0.6, 0.0, 0.0), (0.33, 0.0, 0.0))


def soni_aggradation(n: int = 100, overfeed: float = 4.0, s0: float = 3.56e-3,
                     length: float = 30.0) -> Problem:
    """Aggradation by sediment overfeeding in a sloping flume (Sec. 5.1, the
    Soni case), per unit width: h = 0.05 m, q = 0.02 m^2/s, z = 1.2 - s0 x
    with s0 = 3.56 per mille on [0, 30] m (Eq. Soni0); transport
    q_s = alpha u^beta, alpha = 1.45e-3, beta = 5 (Eq. Soni_qs); porosity 0.4;
    Strickler friction K_s = 49.4 m^(1/3)/s; t_end = 2400 s. Upstream: q = 0.02
    and the solid discharge (1 + overfeed) alpha (q/h)^beta, i.e. the
    equilibrium discharge of the initial uniform flow raised by
    Delta Q_S = overfeed Q_S0 (4 in the paper); downstream: h = 0.05. Both
    ghosts continue the bed slope. CFL 0.9 (not printed for this case)."""
    h0, q0, alpha, beta = 0.05, 0.02, 1.45e-3, 5.0
    x = cell_centres(n, 0.0, length)
    z = 1.2 - s0 * x
    feed = (1.0 + overfeed) * alpha * (q0 / h0) ** beta
    return Problem("soni_aggradation", n, 0.0, length, 0.9, 2400.0, alpha, XI_P04,
                   np.full(n, h0), np.full(n, q0), z, BC_INFLOW_QS, BC_OUTFLOW_HS,
                   (q0, feed, 0.0), (h0, 0.0, 0.0),
                   extra={"ks": 49.4, "beta": beta, "s0": s0, "h0": h0, "q0": q0,
                          "qs0": alpha * (q0 / h0) ** beta})


def lake_at_rest(n: int, seed: int = 7, level: float = 1.0) -> Problem:
    """Still water over a rough bed: z on multiples of 2^-10 in [0, 0.5],
    h = level - z, q = 0, transmissive ends."""
    rng = np.random.default_rng(seed)
    z = rng.integers(0, 512, size=n).astype(np.float64) / 1024.0
    h = level - z
    return Problem("lake_at_rest", n, 0.0, 1.0, 0.9, 1.0, 0.01, XI_P04, h, np.zeros(n), z)


def dam_break(n: int, hL=2.0, hR=1.0, uL=0.0, uR=0.0) -> Problem:
    """Flat-bed fixed-bed dam break on [0, 10] m at 5 m (A_g = 0)."""
    h, q, z = riemann(n, 0.0, 10.0, 5.0, (hL, hL * uL, 0.0), (hR, hR * uR, 0.0))
    return Problem("dam_break", n, 0.0, 10.0, 0.9, 0.5, 0.0, 1.0, h, q, z)


def random_edges(n: int, seed: int, h_range=(0.05, 5.0), fr_range=(-3.0, 3.0),
                 dz_scale=0.3, rel_jump=0.5, g: float = G):
    """Random edge pairs (WL, WR) as [3, n] float64 arrays.

    Left states: h ~ U(h_range), Froude ~ U(fr_range), z ~ U(-0.5, 0.5).
    Right states: left state times (1 + U(-rel_jump, rel_jump)) for h and q,
    z + U(-dz_scale, dz_scale).
    """
    rng = np.random.default_rng(seed)
    hL = rng.uniform(*h_range, size=n)
    frL = rng.uniform(*fr_range, size=n)
    qL = frL * np.sqrt(g * hL) * hL
    zL = rng.uniform(-0.5, 0.5, size=n)
    hR = hL * (1.0 + rng.uniform(-rel_jump, rel_jump, size=n))
    qR = qL * (1.0 + rng.uniform(-rel_jump, rel_jump, size=n)) + 0.01 * rng.standard_normal(n)
    zR = zL + rng.uniform(-dz_scale, dz_scale, size=n)
    return np.stack([hL, qL, zL]), np.stack([hR, qR, zR])


def random_states(n: int, seed: int, h_range=(0.05, 5.0), fr_range=(-3.0, 3.0),
                  g: float = G):
    """Random single states (h, q) with h ~ U(h_range) and Froude ~ U(fr_range)."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(*h_range, size=n)
    fr = rng.uniform(*fr_range, size=n)
    return h, fr * np.sqrt(g * h) * h


@dataclass
class Ensemble:
    """Independent channels laid end to end: channel c owns cells
    offsets[c] .. offsets[c+1]-1 of the concatenated h, q, z arrays."""
    n_cells: np.ndarray  # int64 [C]
    length: np.ndarray   # float64 [C], channel length [m]
    Ag: np.ndarray       # float64 [C]
    h: np.ndarray
    q: np.ndarray
    z: np.ndarray
    xi: float = XI_P04
    cfl: float = 0.9
    t_end: float = 1.0
    g: float = G

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_cells)]).astype(np.int64)

    def channel(self, c: int):
        o = self.offsets
        return self.h[o[c]:o[c + 1]], self.q[o[c]:o[c + 1]], self.z[o[c]:o[c + 1]]


def riemann_ensemble(n_channels: int = 4096, seed: int = 20191210, n_min: int = 1000,
                     n_max: int = 100000, length: float = 10.0) -> Ensemble:
    """Batch of movable-bed Riemann problems: N_c log-uniform in [n_min, n_max];
    h_L, h_R ~ U(0.5, 3) m; u_L, u_R ~ U(-0.5, 1.0) m/s drawn per side;
    z_L = 0, z_R ~ U(-0.3, 0.3) m; A_g ~ U(0.001, 0.02); discontinuity at the
    channel centre; transmissive ends; CFL 0.9, t_end 1 s."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_channels)).astype(np.int64)
    hL, hR = rng.uniform(0.5, 3.0, n_channels), rng.uniform(0.5, 3.0, n_channels)
    uL, uR = rng.uniform(-0.5, 1.0, n_channels), rng.uniform(-0.5, 1.0, n_channels)
    zR = rng.uniform(-0.3, 0.3, n_channels)
    Ag = rng.uniform(0.001, 0.02, n_channels)
    hs, qs, zs = [], [], []
    for c in range(n_channels):
        h, q, z = riemann(int(n[c]), 0.0, length, 0.5 * length, (hL[c], hL[c] * uL[c], 0.0),
                          (hR[c], hR[c] * uR[c], zR[c]))
        hs.append(h)
        qs.append(q)
        zs.append(z)
    return Ensemble(n, np.full(n_channels, length), Ag, np.concatenate(hs), np.concatenate(qs),
                    np.concatenate(zs))


def shard_ensemble(E: "Ensemble", rank: int, world: int) -> "Ensemble":
    """The channels of rank `rank` when the ensemble is split over `world`
    processes (one per GPU; the channels are independent, so no data moves
    between them): longest-processing-time list scheduling of the channels,
    work N_c^2 / length_c (cells times steps, dt ~ dx), largest first onto the
    least-loaded rank (ties to the lower rank), the rank's channels kept in
    their original order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    n = E.n_cells.astype(np.float64)
    work = n * n / E.length
    load = np.zeros(world)
    owner = np.empty(len(n), dtype=np.int64)
    for c in sorted(range(len(n)), key=lambda c: (-work[c], c)):
        r = int(np.argmin(load))
        owner[c] = r
        load[r] += work[c]
    mine = np.flatnonzero(owner == rank)
    o = E.offsets
    cells = np.concatenate([np.arange(o[c], o[c + 1]) for c in mine]) if len(mine) else np.zeros(0, np.int64)
    return Ensemble(E.n_cells[mine].copy(), E.length[mine].copy(), E.Ag[mine].copy(), E.h[cells].copy(),
                    E.q[cells].copy(), E.z[cells].copy(), E.xi, E.cfl, E.t_end, E.g)


def mlp_init(seed: int = 2019, sizes=(7, 128, 128, 128, 128, 9)) -> np.ndarray:
    """Initial surrogate parameters, packed layer by layer (W_l [out][in]
    row-major, then b_l): He-normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in zip(sizes[:-1], sizes[1:]):
        parts.append(rng.standard_normal(o * i) * np.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)
