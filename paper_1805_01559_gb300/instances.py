"""Seeded synthetic C-RAN instances: geometry, path gains, traffic and RRH marginals.

This module is the ONE piece shared by the CUDA path and the FP64 oracle. It
holds none of the method's arithmetic: it draws positions, path gains with
shadowing, per-device traffic and RRH capacities, and nothing downstream of
them (no SINR, no rate, no cost, no Sinkhorn step).  The downlink quantities
it prepares are the ones the paper's model takes as given (Sec. II-A: transmit
power P_j, path gain G_ji, thermal noise N_0, bandwidth W; Sec. II-B: traffic
lambda_i and mean job size 1/mu; Sec. IV: the RRH marginal q).

Channel model (the paper leaves it open; the readings are fixed here):
  * RRHs on a jittered grid: r = floor(sqrt(J)) rows, ceil(J/r) columns, the
    first J cells in row-major order, each RRH at its cell centre plus a
    uniform jitter of +-0.25 cell per axis.
  * devices uniform in the square, or (hot-spot configs) 40% of them drawn
    around 5 centres uniform in the square with an isotropic Gaussian of
    sigma = 0.05 * side, resampled (not clipped) until inside.
  * path loss PL_dB = PL0 + 10 * n * log10(max(d, 10 m)) with PL0 = 30 dB,
    n = 3.5, plus i.i.d. lognormal shadowing X ~ N(0, 8^2) dB per link;
    G = 10^(-(PL_dB + X)/10).
  * P_j = 1 W, W = 20 MHz, N_0 = -174 dBm/Hz + 10 log10(W) + 9 dB noise figure.
  * mu = 1e-6 per bit (mean job size 1 Mbit), so 1/(mu R) is in seconds.
  * traffic lambda_i ~ lognormal(0, sigma), normalised to sum 1.
  * RRH marginal: uniform q_j = sum(lambda)/J (Sec. IV choice (i)) or
    capacity-proportional q_j = kappa_j / sum(kappa) * sum(lambda) with
    kappa_j ~ U[0.5, 1.5].

Every generator takes a numpy ``Generator`` (PCG64) or a seed, so both sides
see bit-identical inputs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

PL0_DB = 30.0
PL_EXPONENT = 3.5
SHADOW_DB = 8.0
D_MIN_M = 10.0
P_TX_W = 1.0
W_HZ = 20e6
NOISE_DBM_HZ = -174.0
NOISE_FIGURE_DB = 9.0
MU_PER_BIT = 1e-6


def noise_power_w(w_hz: float = W_HZ) -> float:
    """Thermal noise power N_0 in watts over the band."""
    dbm = NOISE_DBM_HZ + 10.0 * math.log10(w_hz) + NOISE_FIGURE_DB
    return 10.0 ** ((dbm - 30.0) / 10.0)


def _rng(seed_or_rng) -> np.random.Generator:
    if isinstance(seed_or_rng, np.random.Generator):
        return seed_or_rng
    return np.random.Generator(np.random.PCG64(seed_or_rng))


def rrh_jittered_grid(J: int, side: float, rng) -> np.ndarray:
    """J RRH positions (J x 2, metres) on a jittered grid over [0, side]^2."""
    rng = _rng(rng)
    r = max(1, int(math.isqrt(J)))
    c = -(-J // r)
    cw, ch = side / c, side / r
    k = np.arange(J)
    row, col = k // c, k % c
    jit = rng.uniform(-0.25, 0.25, size=(J, 2))
    x = (col + 0.5 + jit[:, 0]) * cw
    y = (row + 0.5 + jit[:, 1]) * ch
    return np.stack([x, y], axis=1)


def devices_uniform(I: int, side: float, rng) -> np.ndarray:
    rng = _rng(rng)
    return rng.uniform(0.0, side, size=(I, 2))


def devices_hotspot(I: int, side: float, rng, n_spots: int = 5, frac: float = 0.4,
                    sigma_frac: float = 0.05) -> np.ndarray:
    """I device positions; a fraction `frac` sits in Gaussian hot spots."""
    rng = _rng(rng)
    n_hot = int(round(frac * I))
    centres = rng.uniform(0.0, side, size=(n_spots, 2))
    which = rng.integers(0, n_spots, size=n_hot)
    sigma = sigma_frac * side
    hot = centres[which] + rng.normal(0.0, sigma, size=(n_hot, 2))
    bad = np.flatnonzero(((hot < 0) | (hot > side)).any(axis=1))
    while bad.size:
        hot[bad] = centres[which[bad]] + rng.normal(0.0, sigma, size=(bad.size, 2))
        bad = bad[((hot[bad] < 0) | (hot[bad] > side)).any(axis=1)]
    uni = rng.uniform(0.0, side, size=(I - n_hot, 2))
    pos = np.concatenate([hot, uni], axis=0)
    return pos[rng.permutation(I)]


def shadowing_db(I: int, J: int, rng, dtype=np.float32) -> np.ndarray:
    rng = _rng(rng)
    return (rng.standard_normal(size=(I, J), dtype=np.float32) * np.float32(SHADOW_DB)).astype(dtype)


def path_gains(dev_xy: np.ndarray, rrh_xy: np.ndarray, shadow_db: np.ndarray,
               dtype=np.float64, row_chunk: int = 8192) -> np.ndarray:
    """G[i, j]: linear path gain from RRH j to device i (the paper's G_ji)."""
    I, J = dev_xy.shape[0], rrh_xy.shape[0]
    out = np.empty((I, J), dtype=dtype)
    for s in range(0, I, row_chunk):
        e = min(I, s + row_chunk)
        dx = dev_xy[s:e, None, 0] - rrh_xy[None, :, 0]
        dy = dev_xy[s:e, None, 1] - rrh_xy[None, :, 1]
        d = np.maximum(np.sqrt(dx * dx + dy * dy), D_MIN_M)
        pl_db = PL0_DB + 10.0 * PL_EXPONENT * np.log10(d) + shadow_db[s:e].astype(np.float64)
        out[s:e] = np.power(10.0, -pl_db / 10.0)
    return out


def traffic_lognormal(I: int, sigma: float, rng) -> np.ndarray:
    rng = _rng(rng)
    lam = np.exp(sigma * rng.standard_normal(I))
    return lam / lam.sum()


def uniform_marginal(J: int, total: float) -> np.ndarray:
    return np.full(J, total / J)


def capacity_marginal(J: int, total: float, rng) -> np.ndarray:
    rng = _rng(rng)
    kappa = rng.uniform(0.5, 1.5, size=J)
    return kappa / kappa.sum() * total


@dataclasses.dataclass
class Instance:
    """One device-association instance (inputs only)."""
    name: str
    G: np.ndarray            # I x J path gains (row-major), G[i, j] = gain RRH j -> device i
    P: np.ndarray            # J transmit powers (W)
    N0: float                # noise power (W)
    W_hz: float              # bandwidth (Hz)
    mu: float                # 1 / mean job size (1/bit)
    lam: np.ndarray          # I traffic (sum 1) = row marginal p
    q: np.ndarray            # J RRH marginal (sum = sum lam)
    eps_rel: Sequence[float] # eps = eps_rel * median(C)
    tol: float
    max_iter: int
    dev_xy: Optional[np.ndarray] = None
    rrh_xy: Optional[np.ndarray] = None
    shadow_db: Optional[np.ndarray] = None
    side: float = 0.0
    seed: int = 0

    @property
    def I(self) -> int:
        return self.G.shape[0]

    @property
    def J(self) -> int:
        return self.G.shape[1]


def make_instance(name: str, I: int, J: int, side: float, seed: int, *, hotspot: bool,
                  traffic_sigma: float, marginal: str, eps_rel=(0.05,), tol: float = 1e-6,
                  max_iter: int = 2000, dtype=np.float64, keep_geometry: bool = False) -> Instance:
    """Draw one instance. Streams are split so each part is independent of the others."""
    root = np.random.SeedSequence(seed)
    s_rrh, s_dev, s_sh, s_lam, s_q = [np.random.Generator(np.random.PCG64(s)) for s in root.spawn(5)]
    rrh = rrh_jittered_grid(J, side, s_rrh)
    dev = devices_hotspot(I, side, s_dev) if hotspot else devices_uniform(I, side, s_dev)
    sh = shadowing_db(I, J, s_sh)
    G = path_gains(dev, rrh, sh, dtype=dtype)
    lam = traffic_lognormal(I, traffic_sigma, s_lam)
    if marginal == "uniform":
        q = uniform_marginal(J, lam.sum())
    elif marginal == "capacity":
        q = capacity_marginal(J, lam.sum(), s_q)
    else:
        raise ValueError(marginal)
    return Instance(name=name, G=G, P=np.full(J, P_TX_W), N0=noise_power_w(), W_hz=W_HZ,
                    mu=MU_PER_BIT, lam=lam, q=q, eps_rel=tuple(eps_rel), tol=tol,
                    max_iter=max_iter, dev_xy=dev if keep_geometry else None,
                    rrh_xy=rrh if keep_geometry else None,
                    shadow_db=sh if keep_geometry else None, side=side, seed=seed)


def config1(seed: int = 0, dtype=np.float64) -> Instance:
    """1000 devices uniform in 1 km^2, 50 RRHs, lognormal(0,1) traffic, uniform q."""
    return make_instance("c1_1000x50", 1000, 50, 1000.0, seed, hotspot=False, traffic_sigma=1.0,
                         marginal="uniform", eps_rel=(0.05,), dtype=dtype)


def config2(seed: int = 0, dtype=np.float32) -> Instance:
    """50,000 devices in 4 km^2 with 5 hot spots (40%), 800 RRHs, capacity q, eps sweep."""
    return make_instance("c2_50000x800", 50_000, 800, 2000.0, seed, hotspot=True,
                         traffic_sigma=1.5, marginal="capacity", eps_rel=(0.1, 0.03, 0.01),
                         dtype=dtype)


def config3_shapes(n: int = 256, base_seed: int = 0):
    """(I, J, seed) of the ragged batch: I ~ U{2000..60000}, J ~ U{64..1024}."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([base_seed, 3])))
    Is = rng.integers(2000, 60001, size=n)
    Js = rng.integers(64, 1025, size=n)
    return [(int(Is[k]), int(Js[k]), base_seed + k) for k in range(n)]


def config3_cell(I: int, J: int, seed: int, dtype=np.float32) -> Instance:
    """One batched cell: channel and traffic as config 1 (1 km^2, uniform devices, uniform q)."""
    return make_instance(f"c3_{I}x{J}_s{seed}", I, J, 1000.0, seed, hotspot=False,
                         traffic_sigma=1.0, marginal="uniform", eps_rel=(0.05,), dtype=dtype)


def config4(seed: int = 0, dtype=np.float32, I: int = 400_000, J: int = 4096) -> Instance:
    """400,000 devices in 16 km^2 with hot spots, 4096 RRHs, capacity q."""
    return make_instance(f"c4_{I}x{J}", I, J, 4000.0, seed, hotspot=True, traffic_sigma=1.5,
                         marginal="capacity", eps_rel=(0.05,), dtype=dtype)


def subsample(inst: Instance, I_sub: int, J_sub: int, seed: int = 1) -> Instance:
    """Seeded random sub-instance (rows and columns), marginals renormalised to balance."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 4])))
    rows = np.sort(rng.choice(inst.I, size=I_sub, replace=False))
    cols = np.sort(rng.choice(inst.J, size=J_sub, replace=False))
    lam = inst.lam[rows] / inst.lam[rows].sum()
    q = inst.q[cols] / inst.q[cols].sum()
    return dataclasses.replace(inst, name=f"{inst.name}_sub{I_sub}x{J_sub}",
                               G=np.ascontiguousarray(inst.G[np.ix_(rows, cols)]),
                               P=inst.P[cols], lam=lam, q=q, dev_xy=None, rrh_xy=None,
                               shadow_db=None)


# ----------------------------------------------------------------------------------------------
# Serving workload: cells whose devices move between time instances (shadowing fixed per link).
# ----------------------------------------------------------------------------------------------
SERVE_I_CHOICES = (5_000, 20_000, 80_000)
SERVE_J_CHOICES = (128, 512, 1024)


def serving_cell_shapes(n_cells: int = 64, base_seed: int = 0):
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([base_seed, 5])))
    Is = rng.choice(SERVE_I_CHOICES, size=n_cells)
    Js = rng.choice(SERVE_J_CHOICES, size=n_cells)
    return [(int(Is[k]), int(Js[k]), base_seed + 1000 + k) for k in range(n_cells)]


@dataclasses.dataclass
class MobileCell:
    """A serving cell: fixed RRHs and shadowing, devices moving with constant velocity."""
    I: int
    J: int
    side: float
    rrh_xy: np.ndarray
    dev_xy: np.ndarray
    vel: np.ndarray
    shadow_db: np.ndarray
    lam: np.ndarray
    q: np.ndarray
    seed: int

    def advance(self, dt: float) -> None:
        """Move every device by vel*dt, reflecting at the square's walls."""
        pos = self.dev_xy + self.vel * dt
        for ax in range(2):
            p = np.mod(pos[:, ax], 2.0 * self.side)
            refl = p > self.side
            p[refl] = 2.0 * self.side - p[refl]
            flip = (np.floor_divide(self.dev_xy[:, ax] + self.vel[:, ax] * dt, self.side)
                    .astype(np.int64) % 2) == 1
            self.vel[flip, ax] = -self.vel[flip, ax]
            pos[:, ax] = p
        self.dev_xy = pos

    def gains(self, dtype=np.float32) -> np.ndarray:
        return path_gains(self.dev_xy, self.rrh_xy, self.shadow_db, dtype=dtype)


def serving_cell(I: int, J: int, seed: int, side: float = 1000.0) -> MobileCell:
    root = np.random.SeedSequence(seed)
    s_rrh, s_dev, s_sh, s_lam, s_v = [np.random.Generator(np.random.PCG64(s)) for s in root.spawn(5)]
    rrh = rrh_jittered_grid(J, side, s_rrh)
    dev = devices_uniform(I, side, s_dev)
    speed = s_v.uniform(1.0, 30.0, size=I)
    heading = s_v.uniform(0.0, 2.0 * math.pi, size=I)
    vel = np.stack([speed * np.cos(heading), speed * np.sin(heading)], axis=1)
    sh = shadowing_db(I, J, s_sh)
    lam = traffic_lognormal(I, 1.0, s_lam)
    return MobileCell(I=I, J=J, side=side, rrh_xy=rrh, dev_xy=dev, vel=vel, shadow_db=sh,
                      lam=lam, q=uniform_marginal(J, lam.sum()), seed=seed)


def poisson_arrivals(rate_hz: float, duration_s: float, n_cells: int, seed: int = 0):
    """Arrival times (s) and the cell index of each request."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 6])))
    n = rng.poisson(rate_hz * duration_s)
    t = np.sort(rng.uniform(0.0, duration_s, size=n))
    cells = rng.integers(0, n_cells, size=n)
    return t, cells


# ----------------------------------------------------------------------------------------------
# Large instances in row blocks (each block's shadowing from its own seed), so that the gains
# can be drawn in parallel and streamed to the device block by block.
# ----------------------------------------------------------------------------------------------
@dataclasses.dataclass
class BlockedInstance:
    """An instance whose gains are produced block by block (gains_block)."""
    name: str
    I: int
    J: int
    side: float
    seed: int
    block: int
    rrh_xy: np.ndarray
    dev_xy: np.ndarray
    P: np.ndarray
    N0: float
    W_hz: float
    mu: float
    lam: np.ndarray
    q: np.ndarray

    @property
    def nblocks(self) -> int:
        return (self.I + self.block - 1) // self.block

    def gains_block(self, b: int, dtype=np.float32) -> np.ndarray:
        r0, r1 = b * self.block, min(self.I, (b + 1) * self.block)
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([self.seed, 7, b])))
        sh = shadowing_db(r1 - r0, self.J, rng)
        return path_gains(self.dev_xy[r0:r1], self.rrh_xy, sh, dtype=dtype)


def config4_blocked(seed: int = 0, I: int = 400_000, J: int = 4096, block: int = 8192) -> BlockedInstance:
    """The 400,000 x 4,096 configuration (16 km^2, hot spots, capacity q) in row blocks."""
    root = np.random.SeedSequence(seed)
    s_rrh, s_dev, _, s_lam, s_q = [np.random.Generator(np.random.PCG64(s)) for s in root.spawn(5)]
    side = 4000.0
    rrh = rrh_jittered_grid(J, side, s_rrh)
    dev = devices_hotspot(I, side, s_dev)
    lam = traffic_lognormal(I, 1.5, s_lam)
    q = capacity_marginal(J, lam.sum(), s_q)
    return BlockedInstance(name=f"c4_{I}x{J}", I=I, J=J, side=side, seed=seed, block=block, rrh_xy=rrh,
                           dev_xy=dev, P=np.full(J, P_TX_W), N0=noise_power_w(), W_hz=W_HZ, mu=MU_PER_BIT,
                           lam=lam, q=q)


@dataclasses.dataclass
class PolicyCell:
    """A cell of the uniform-traffic policy comparison (Sec. IV): J RRHs on a jittered grid,
    N devices uniform in the square, distance-only path loss (no shadowing), equal traffic
    per device (unit total; the comparison scales it)."""
    G: np.ndarray        # N x J gains (float32)
    P: np.ndarray        # J powers
    N0: float
    W_hz: float
    mu: float
    dev_xy: np.ndarray   # N x 2 (float32)
    rrh_xy: np.ndarray   # J x 2 (float32)
    lam: np.ndarray      # N, equal, sum 1
    side: float


def policy_cell(N: int, seed: int, J: int = 25, side: float = 1000.0) -> PolicyCell:
    rng = _rng(np.random.SeedSequence([seed, 11, N]))
    rrh = rrh_jittered_grid(J, side, rng).astype(np.float32)
    dev = devices_uniform(N, side, rng).astype(np.float32)
    G = path_gains(dev.astype(np.float64), rrh.astype(np.float64), np.zeros((N, J), np.float32), dtype=np.float32)
    return PolicyCell(G=G, P=np.full(J, P_TX_W), N0=noise_power_w(), W_hz=W_HZ, mu=MU_PER_BIT, dev_xy=dev,
                      rrh_xy=rrh, lam=np.full(N, 1.0 / N), side=side)
