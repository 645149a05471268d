"""Seeded synthetic inputs for the Poisson-lognormal MAP solve.

This module builds the data the solver consumes -- galaxy counts N, the
completeness w, the mean count nbar, the prior mean mu and a tabulated power
spectrum P(k) -- and the true log-density s_true they were drawn from.  It is
deliberately independent of both the CUDA library and the CPU oracle: it holds
none of the solver's arithmetic (no prior operator, no gradient, no Hessian),
only the generative model of the paper's mock catalogues:

* The paper draws its mocks as a Poisson sample of a density field with an
  expected count nbar * w_i * (1 + delta_i) per cell (Sec. 2.1, the likelihood
  equation and the definition of <N>) and a lognormal density
  1 + delta = exp(s) (Sec. 2.3).  Its Millennium-run density field is not
  available, so a Gaussian random field G with power spectrum
  P(k) = A k / (1 + (k/0.02)^2)^1.4 stands in for the log-density:
  s_true = G - sigma_G^2 / 2, so that <1 + delta> = 1 (Sec. 2.3, the mean-field
  equation for mu).
* Randomness comes from Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel
  random numbers: as easy as 1, 2, 3", SC'11), keyed by (seed, mock id) and
  addressed by (cell index, stream tag, draw index, 0).  Stream tags:
  0 = Gaussian white noise, 1 = Poisson draws, 2 = angular mask, 3 = batch
  parameters.  Gaussians use the Box-Muller transform; Poisson counts use
  inversion by sequential search on pieces of mean <= 30 (a Poisson variable of
  mean lam is the sum of m independent ones of mean lam/m).
* The counts are generated once on the host and the same int32 buffer is
  handed to every consumer, so they are bit-identical by construction.

Discrete conventions (shared by the data model and the solver's prior):
the unnormalised forward DFT diagonalises the prior covariance with eigenvalue
lambda_k = P(|k|) n^3 / L^3 (per-cell variance units), |k| = (2 pi / L) |m| with
integer mode m in [-n/2, n/2); sigma_G^2 = n^-3 sum_{k != 0} lambda_k fixes A.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al. 2011): 10 rounds of a multiply-hi/lo S-box with
# a Weyl-sequence key schedule.
# ---------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)
_SHIFT32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32-10 block function on arrays of 32-bit counters.

    Returns the four 32-bit output words (as uint64 arrays holding values
    < 2^32).  Round: (hi0, lo0) = M0*c0, (hi1, lo1) = M1*c2, new counter
    (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by the Weyl
    constants between rounds.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    ka, kb = k0 & 0xFFFFFFFF, k1 & 0xFFFFFFFF
    for r in range(10):
        if r:
            ka = (ka + _PHILOX_W0) & 0xFFFFFFFF
            kb = (kb + _PHILOX_W1) & 0xFFFFFFFF
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> _SHIFT32, p0 & _MASK32
        hi1, lo1 = p1 >> _SHIFT32, p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(ka), lo1,
                          hi0 ^ c3 ^ np.uint64(kb), lo0)
    return c0, c1, c2, c3


def _u53(a, b):
    """Two 32-bit words -> a double uniform on the open interval (0, 1)."""
    hi = (a >> np.uint64(5)).astype(np.float64)   # 27 bits
    lo = (b >> np.uint64(6)).astype(np.float64)   # 26 bits
    return (hi * 67108864.0 + lo + 0.5) / 9007199254740992.0


TAG_NOISE, TAG_POISSON, TAG_MASK, TAG_BATCH = 0, 1, 2, 3


def uniform_pair(index, tag: int, draw: int, seed: int, mock_id: int):
    """Two independent U(0,1) doubles per element of `index`."""
    index = np.asarray(index, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32_10(index, tag, draw, 0, seed, mock_id)
    return _u53(w0, w1), _u53(w2, w3)


def white_noise(n: int, seed: int, mock_id: int = 0) -> np.ndarray:
    """Unit-variance Gaussian white noise on an n^3 grid ([z][y][x])."""
    cells = np.arange(n ** 3, dtype=np.uint64)
    u1, u2 = uniform_pair(cells, TAG_NOISE, 0, seed, mock_id)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return z.reshape(n, n, n)


# ---------------------------------------------------------------------------
# Power spectrum of the synthetic log-density and its tabulation.
# ---------------------------------------------------------------------------

def pk_shape(k):
    """Unnormalised P(k) = k / (1 + (k/0.02)^2)^1.4, k in h/Mpc."""
    k = np.asarray(k, dtype=np.float64)
    return k / (1.0 + (k / 0.02) ** 2) ** 1.4


def _mode_m2(n: int) -> np.ndarray:
    """|m|^2 for every mode of the full n^3 DFT grid, m_i in [-n/2, n/2)."""
    m = np.arange(n)
    m = np.where(m < (n + 1) // 2, m, m - n).astype(np.float64)
    return m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2


def amplitude_for_sigma(n: int, box: float, sigma_G: float) -> float:
    """A such that n^-3 sum_{k != 0} P(|k|) n^3 / L^3 = sigma_G^2."""
    kk = (2.0 * np.pi / box) * np.sqrt(_mode_m2(n))
    shape = pk_shape(kk)
    shape.flat[0] = 0.0
    return sigma_G ** 2 * box ** 3 / float(shape.sum())


def pk_table(n: int, box: float, A: float, nbins: int = 512):
    """Log-spaced (k, P) table from 0.5 k_f to 1.01 sqrt(3) k_Nyquist."""
    kf = 2.0 * np.pi / box
    kmax = 1.01 * math.sqrt(3.0) * np.pi * n / box
    k = np.exp(np.linspace(math.log(0.5 * kf), math.log(kmax), nbins))
    return k, A * pk_shape(k)


def gaussian_field(n: int, box: float, A: float, seed: int,
                   mock_id: int = 0) -> np.ndarray:
    """Gaussian field with covariance eigenvalues lambda_k = A*shape n^3/L^3.

    G = IDFT(DFT(eps) * sqrt(lambda_k)) with eps white noise; the DC mode has
    lambda_0 = 0, so G has zero mean.  Uses numpy's FFT (data synthesis only).
    """
    eps = white_noise(n, seed, mock_id)
    kk = (2.0 * np.pi / box) * np.sqrt(_mode_m2(n))[:, :, : n // 2 + 1]
    lam = A * pk_shape(kk) * n ** 3 / box ** 3
    lam[0, 0, 0] = 0.0
    E = np.fft.rfftn(eps)
    return np.fft.irfftn(E * np.sqrt(lam), s=(n, n, n), axes=(0, 1, 2))


def poisson_counts(lam: np.ndarray, seed: int, mock_id: int = 0,
                   piece: float = 30.0) -> np.ndarray:
    """Poisson(lam) per cell by inversion on pieces of mean <= `piece`.

    Cell i is split into m_i = max(1, ceil(lam_i / piece)) independent pieces
    of mean lam_i / m_i; piece j of cell i uses the uniform from counter
    (i, TAG_POISSON, j, 0).  Each piece is the smallest k with CDF(k) >= u.
    """
    shape = lam.shape
    lam = np.ascontiguousarray(lam, dtype=np.float64).ravel()
    if np.any(~np.isfinite(lam)) or np.any(lam < 0):
        raise ValueError("Poisson means must be finite and >= 0")
    m = np.maximum(1, np.ceil(lam / piece)).astype(np.int64)
    lp = lam / m
    out = np.zeros(lam.size, dtype=np.int64)
    for j in range(int(m.max()) if lam.size else 0):
        cells = np.nonzero(m > j)[0]
        u, _ = uniform_pair(cells.astype(np.uint64), TAG_POISSON, j,
                            seed, mock_id)
        lj = lp[cells]
        p = np.exp(-lj)
        cdf = p.copy()
        k_of = np.zeros(cells.size, dtype=np.int64)
        act = np.nonzero(u > cdf)[0]
        k = 0
        while act.size and k < 1000:
            k += 1
            p[act] *= lj[act] / k
            cdf[act] += p[act]
            k_of[act] = k
            act = act[u[act] > cdf[act]]
        out[cells] += k_of
    if out.max(initial=0) > np.iinfo(np.int32).max:
        raise OverflowError("count exceeds int32")
    return out.astype(np.int32).reshape(shape)


def cell_centres(n: int, box: float):
    """Distance components of cell centres (i + 1/2) L / n from the box centre."""
    c = (np.arange(n) + 0.5) * box / n - 0.5 * box
    return c[:, None, None], c[None, :, None], c[None, None, :]   # dz, dy, dx


def radial_masked_selection(n: int, box: float, r0: float = 200.0,
                            mask_fraction: float = 0.2, seed: int = 1,
                            mock_id: int = 0, ncos: int = 16,
                            nphi: int = 32) -> np.ndarray:
    """w(r) = exp(-(r/r0)^2) about the box centre, zero in masked patches.

    The sky is cut into ncos x nphi equal-area patches (uniform bins in
    cos(theta) and phi, theta from the z axis); floor(mask_fraction * npatch)
    of them, the ones with the smallest Philox keys, are masked.
    """
    dz, dy, dx = cell_centres(n, box)
    dz, dy, dx = np.broadcast_arrays(dz, dy, dx)
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    w = np.exp(-(r / r0) ** 2)
    cos_t = np.clip(dz / np.where(r > 0, r, 1.0), -1.0, 1.0)
    phi = np.mod(np.arctan2(dy, dx), 2.0 * np.pi)
    ic = np.minimum(ncos - 1, np.floor((cos_t + 1.0) * 0.5 * ncos)).astype(int)
    ip = np.minimum(nphi - 1, np.floor(phi / (2.0 * np.pi) * nphi)).astype(int)
    patch = ic * nphi + ip
    npatch = ncos * nphi
    keys = philox4x32_10(np.arange(npatch, dtype=np.uint64), TAG_MASK, 0, 0,
                         seed, mock_id)
    key64 = (keys[0] << _SHIFT32) | keys[1]
    masked = np.argsort(key64, kind="stable")[: int(math.floor(mask_fraction * npatch))]
    is_masked = np.zeros(npatch, dtype=bool)
    is_masked[masked] = True
    w = np.where(is_masked[patch] & (r > 0), 0.0, w)
    return w


# ---------------------------------------------------------------------------
# Workload definitions.
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class MockSpec:
    name: str
    n: int
    box: float              # Mpc/h
    sigma_G: float
    nbar: float             # mean count per cell
    selection: str = "uniform"   # "uniform" (w = 1) or "radial_masked"
    seed: int = 1
    mock_id: int = 0
    nbins: int = 512


@dataclass
class Mock:
    spec: MockSpec
    N: np.ndarray                 # int32 [n][n][n]
    w: Optional[np.ndarray]       # float64 [n][n][n] or None (w = 1)
    nbar: float
    mu: float
    k_tab: np.ndarray
    P_tab: np.ndarray
    A: float
    s_true: np.ndarray = field(repr=False)

    @property
    def n(self) -> int:
        return self.spec.n

    @property
    def box(self) -> float:
        return self.spec.box


WORKLOADS = {
    # 32^3, 200 Mpc/h, sigma_G = 1, nbar = 2 per cell, w = 1, seed 1.
    "plain32": MockSpec("plain32", 32, 200.0, 1.0, 2.0),
    # 128^3, 500 Mpc/h, sigma_G = 1.5, nbar = 0.5, radial selection + mask.
    "selection128": MockSpec("selection128", 128, 500.0, 1.5, 0.5, "radial_masked"),
    # 256^3, 500 Mpc/h, sigma_G = 1.8, nbar = 1, w = 1 (production size).
    "production256": MockSpec("production256", 256, 500.0, 1.8, 1.0),
    # Differentiation workloads: 128^3 / 500 and 32^3 / 200, sigma_G = 1.2.
    "adjoint128": MockSpec("adjoint128", 128, 500.0, 1.2, 1.0),
    "adjoint32": MockSpec("adjoint32", 32, 200.0, 1.2, 1.0),
}


def make_mock(spec: MockSpec) -> Mock:
    """Draw the counts, selection and prior table for one workload."""
    n, box = spec.n, spec.box
    A = amplitude_for_sigma(n, box, spec.sigma_G)
    G = gaussian_field(n, box, A, spec.seed, spec.mock_id)
    s_true = G - 0.5 * spec.sigma_G ** 2
    if spec.selection == "uniform":
        w = None
        lam = spec.nbar * np.exp(s_true)
    elif spec.selection == "radial_masked":
        w = radial_masked_selection(n, box, seed=spec.seed, mock_id=spec.mock_id)
        lam = spec.nbar * w * np.exp(s_true)
    else:
        raise ValueError(f"unknown selection {spec.selection!r}")
    N = poisson_counts(lam, spec.seed, spec.mock_id)
    k_tab, P_tab = pk_table(n, box, A, spec.nbins)
    return Mock(spec=spec, N=N, w=w, nbar=spec.nbar,
                mu=-0.5 * spec.sigma_G ** 2, k_tab=k_tab, P_tab=P_tab, A=A,
                s_true=s_true)


def batch_specs(seed_base: int = 1):
    """64 independent mocks of uneven size: 16 x 64^3, 32 x 96^3, 16 x 128^3.

    Each has its own seed; sigma_G ~ U[0.8, 1.8] and nbar log-uniform in
    [0.2, 2] (drawn from Philox, stream TAG_BATCH); L = 3.90625 n Mpc/h.
    """
    sizes = [64] * 16 + [96] * 32 + [128] * 16
    ids = np.arange(len(sizes), dtype=np.uint64)
    u1, u2 = uniform_pair(ids, TAG_BATCH, 0, seed_base, 0)
    specs = []
    for i, n in enumerate(sizes):
        sig = 0.8 + 1.0 * float(u1[i])
        nbar = math.exp(math.log(0.2) + (math.log(2.0) - math.log(0.2)) * float(u2[i]))
        specs.append(MockSpec(f"batch{i:02d}_{n}", n, 3.90625 * n, sig, nbar,
                              "uniform", seed=seed_base + i, mock_id=i))
    return specs


def bias_table(n: int, box: float, b0: float = 1.5, tilt: float = 0.1, k_ref: float = 0.1,
               nb: int = 32):
    """A scale-dependent linear bias table covering an n^3 grid of side `box`:
    b(k) = b0 (k / k_ref)^tilt (k in h/Mpc), the galaxy-to-matter amplitude
    ratio sqrt(P_g / P_M) of a mildly scale-dependent tracer."""
    kf = 2 * math.pi / box
    k = np.exp(np.linspace(math.log(0.5 * kf), math.log(1.02 * math.sqrt(3) * math.pi * n / box), nb))
    return k, b0 * (k / k_ref) ** tilt


def small_spec(n: int, box: float = 200.0, sigma_G: float = 1.0,
               nbar: float = 2.0, selection: str = "uniform", seed: int = 1,
               nbins: int = 512) -> MockSpec:
    """A small workload of the same family, for tests."""
    return MockSpec(f"small{n}", n, box, sigma_G, nbar, selection, seed, 0, nbins)


def digest(buf: np.ndarray) -> str:
    """SHA-256 of a buffer's bytes, to record which input a run used."""
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(buf).tobytes()).hexdigest()[:16]


__all__ = [
    "philox4x32_10", "uniform_pair", "white_noise", "pk_shape",
    "amplitude_for_sigma", "pk_table", "gaussian_field", "poisson_counts",
    "radial_masked_selection", "MockSpec", "Mock", "WORKLOADS", "make_mock",
    "batch_specs", "small_spec", "bias_table", "digest", "replace",
]
