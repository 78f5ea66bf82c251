"""Seeded synthetic tensor streams shared by the FP64 oracle tests and the GPU path.

This module only draws inputs. It holds none of the decomposition's arithmetic
(no SVD, projection, Gram matrix or truncation), so the oracle and the CUDA
path can both consume its arrays without sharing any of the method.

Every generator is a pure function of (seed, item index): item ``m`` of a
stream is drawn from ``numpy.random.default_rng([seed, m])`` (PCG64), so any
item of any increment can be regenerated on its own, on any machine.

The streams stand in for the paper's data sets (Section 4, Table 1: PDE
simulations and cyber-physical sensor streams), which are not available here:

* ``gaussian_bumps``   — 16^3 items, sums of 5 separable Gaussian bumps plus
  N(0, 1e-6) noise (the smallest case, FP64).
* ``spectral_field``   — 64^3 (or n^3) snapshots of a scalar field made of all
  Fourier modes 0 < |k| <= K with |k|^slope amplitudes and per-stream uniform
  random phases, advected by a constant velocity between snapshots; built by an
  inverse FFT of a Hermitian spectrum (the 3D turbulence-like stream).
* ``multivar_field``   — 5 variables x 48^3 from the same spectral generator,
  independent phases per variable and a per-variable scale in U(0.1, 10).
* ``chebyshev_sensor`` — 24^5 items, sums of 20 separable products of random
  Chebyshev series of degree <= 6 plus 0.01 N(0, 1) noise. The noise comes from
  a counter-based generator (SplitMix64 words, Box-Muller) so that the device
  generator of the library can draw the same stream at HBM rate.
* ``graded_stream``    — two-way items whose mode-1 unfolding has singular
  values graded geometrically over many decades (a numerical stress case for
  tight tolerances, not a stand-in for a data set).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_bumps",
    "spectral_field",
    "multivar_field",
    "chebyshev_sensor",
    "increment_sizes",
    "halfspace_wavevectors",
    "graded_stream",
    "chebyshev_coefficients",
    "counter_normals",
]


def _item_rng(seed: int, m: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(m)])


# ---------------------------------------------------------------------------
# Smallest case: separable Gaussian bumps
# ---------------------------------------------------------------------------

def gaussian_bumps(seed: int, first: int, count: int, n: int = 16, terms: int = 5,
                   noise_std: float = 1e-6) -> np.ndarray:
    """Items ``first .. first+count-1`` of the Gaussian-bump stream, float64 [count, n, n, n].

    item = sum_q a_q g(x; c1q, w1q) g(y; c2q, w2q) g(z; c3q, w3q) + N(0, noise_std^2),
    g(t; c, w) = exp(-(t - c)^2 / (2 w^2)), grid t_i = i / (n - 1),
    c ~ U(0, 1), w ~ U(0.05, 0.3), a ~ N(0, 1).
    """
    t = np.arange(n, dtype=np.float64) / (n - 1)
    out = np.empty((count, n, n, n), dtype=np.float64)
    for j in range(count):
        rng = _item_rng(seed, first + j)
        c = rng.uniform(0.0, 1.0, size=(terms, 3))
        w = rng.uniform(0.05, 0.3, size=(terms, 3))
        a = rng.normal(size=terms)
        g = np.exp(-((t[None, None, :] - c[:, :, None]) ** 2) / (2.0 * w[:, :, None] ** 2))
        item = np.einsum("q,qi,qj,qk->ijk", a, g[:, 0], g[:, 1], g[:, 2])
        item += noise_std * rng.normal(size=item.shape)
        out[j] = item
    return out


# ---------------------------------------------------------------------------
# Spectral (turbulence-like) field
# ---------------------------------------------------------------------------

def halfspace_wavevectors(K: int) -> np.ndarray:
    """Integer wave vectors 0 < |k| <= K, one representative of each +-k pair, int64 [M, 3]."""
    r = np.arange(-K, K + 1)
    kx, ky, kz = np.meshgrid(r, r, r, indexing="ij")
    k = np.stack([kx.ravel(), ky.ravel(), kz.ravel()], axis=1)
    k2 = (k ** 2).sum(1)
    keep = (k2 > 0) & (k2 <= K * K)
    half = (k[:, 0] > 0) | ((k[:, 0] == 0) & (k[:, 1] > 0)) | (
        (k[:, 0] == 0) & (k[:, 1] == 0) & (k[:, 2] > 0))
    return k[keep & half].astype(np.int64)


class _SpectralStream:
    """Fixed per-stream spectrum: amplitudes, phases and advection velocity."""

    def __init__(self, seed: int, n: int, K: int, slope: float, speed: float,
                 stream_tag: int = 0):
        self.n = n
        self.k = halfspace_wavevectors(K)
        kk = np.sqrt((self.k.astype(np.float64) ** 2).sum(1))
        rng = np.random.default_rng([int(seed), 1_000_003, int(stream_tag)])
        amp = kk ** slope
        # a cosine of amplitude a has mean square a^2 / 2: normalise the rms to 1
        amp /= np.sqrt(0.5 * (amp ** 2).sum())
        self.amp = amp
        self.phi = rng.uniform(0.0, 2.0 * np.pi, size=len(kk))
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        self.v = v * speed / n  # `speed` grid cells per snapshot (domain length 1)

    def snapshot(self, t: float) -> np.ndarray:
        n = self.n
        phase = self.phi - 2.0 * np.pi * (self.k @ (self.v * t))
        c = 0.5 * self.amp * np.exp(1j * phase)
        spec = np.zeros((n, n, n), dtype=np.complex128)
        idx = self.k % n
        nidx = (-self.k) % n
        np.add.at(spec, (idx[:, 0], idx[:, 1], idx[:, 2]), c)
        np.add.at(spec, (nidx[:, 0], nidx[:, 1], nidx[:, 2]), np.conj(c))
        return np.fft.ifftn(spec).real * float(n) ** 3


def spectral_field(seed: int, first: int, count: int, n: int = 64, K: int = 16,
                   slope: float = -5.0 / 3.0, speed: float = 1.0,
                   dtype=np.float32) -> np.ndarray:
    """Snapshots ``first .. first+count-1`` of one advected spectral field, [count, n, n, n].

    f(x, t) = sum_{k in K} A |k|^slope cos(2 pi k.(x - v t) + phi_k) over the
    half-space representatives of 0 < |k| <= K, x_i = i / n, phi ~ U(0, 2 pi)
    fixed per stream, v a fixed random direction with |v| = `speed` grid cells
    per snapshot, A normalising the rms to 1.
    """
    s = _SpectralStream(seed, n, K, slope, speed)
    out = np.empty((count, n, n, n), dtype=dtype)
    for j in range(count):
        out[j] = s.snapshot(float(first + j))
    return out


def multivar_field(seed: int, first: int, count: int, n: int = 48, nvar: int = 5,
                   K: int = 16, dtype=np.float32) -> np.ndarray:
    """Items of the multi-variable stream, [count, nvar, n, n, n].

    Each variable is an independent spectral field (own phases and velocity)
    times a per-stream scale s_v ~ U(0.1, 10).
    """
    rng = np.random.default_rng([int(seed), 2_000_003])
    scale = rng.uniform(0.1, 10.0, size=nvar)
    streams = [_SpectralStream(seed, n, K, -5.0 / 3.0, 1.0, stream_tag=v + 1)
               for v in range(nvar)]
    out = np.empty((count, nvar, n, n, n), dtype=dtype)
    for j in range(count):
        for v in range(nvar):
            out[j, v] = scale[v] * streams[v].snapshot(float(first + j))
    return out


def increment_sizes(seed: int, count: int, low: int = 1, high: int = 64) -> np.ndarray:
    """Uneven increment sizes N_k ~ U{low..high} for one stream, int64 [count]."""
    rng = np.random.default_rng([int(seed), 3_000_017])
    return rng.integers(low, high + 1, size=count).astype(np.int64)


# ---------------------------------------------------------------------------
# Smooth sensor-grid responses: Chebyshev products
# ---------------------------------------------------------------------------

def _chebyshev_basis(n: int, degree: int) -> np.ndarray:
    """T_j(x_i) on a uniform grid of n points in [-1, 1], float64 [degree + 1, n]."""
    x = np.linspace(-1.0, 1.0, n)
    T = np.empty((degree + 1, n))
    T[0] = 1.0
    if degree >= 1:
        T[1] = x
    for j in range(2, degree + 1):
        T[j] = 2.0 * x * T[j - 1] - T[j - 2]
    return T


_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _mix64(z: np.ndarray) -> np.ndarray:
    """The output function of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): a bijective mix of
    64-bit words by two xor-shift-multiply steps and a final xor-shift (wrapping uint64 arithmetic)."""
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def counter_normals(seed: int, item: int, count: int) -> np.ndarray:
    """Standard normal draws 0 .. count-1 of one item, float64, from a counter-based generator that a
    device kernel can evaluate element by element.

    The item's base word is b = mix64(seed * 2^32 + item); word k is mix64(b + (k + 1) * gamma), the k-th
    output of a SplitMix64 sequence started at b (gamma = 0x9E3779B97F4A7C15). Word k gives draws 2k and
    2k + 1 by the Box-Muller transform: u1 from its bits 40..63 and u2 from its bits 8..31, each
    (integer + 1/2) / 2^24, then sqrt(-2 ln u1) cos(2 pi u2) and sqrt(-2 ln u1) sin(2 pi u2).
    """
    with np.errstate(over="ignore"):
        b = _mix64(np.array([(int(seed) << 32) + int(item)], dtype=np.uint64))[0]
        k = np.arange((count + 1) // 2, dtype=np.uint64)
        w = _mix64(b + (k + np.uint64(1)) * _GAMMA)
    u1 = ((w >> np.uint64(40)).astype(np.float64) + 0.5) * 2.0 ** -24
    u2 = (((w >> np.uint64(8)) & np.uint64(0xFFFFFF)).astype(np.float64) + 0.5) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * len(k))
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def chebyshev_coefficients(seed: int, first: int, count: int, d: int = 5, terms: int = 20,
                           degree: int = 6) -> np.ndarray:
    """The random coefficients c_{qmj} ~ N(0, 1) of items first .. first+count-1 of the Chebyshev
    sensor stream, float64 [count, terms, d, degree + 1] (item m drawn from default_rng([seed, m]))."""
    out = np.empty((count, terms, d, degree + 1))
    for j in range(count):
        out[j] = _item_rng(seed, first + j).normal(size=(terms, d, degree + 1))
    return out


def chebyshev_sensor(seed: int, first: int, count: int, n: int = 24, d: int = 5,
                     terms: int = 20, degree: int = 6, noise_std: float = 0.01,
                     dtype=np.float32) -> np.ndarray:
    """Items of the Chebyshev sensor stream, [count] + [n] * d.

    item = sum_{q=1..terms} prod_{m=1..d} (sum_{j=0..degree} c_{qmj} T_j(x_m))
           + noise_std * z,  c ~ N(0, 1) (chebyshev_coefficients), z the counter-based standard
    normal draws of counter_normals in C order of the item's elements; x on n uniform points of [-1, 1].
    """
    T = _chebyshev_basis(n, degree)
    out = np.empty((count,) + (n,) * d, dtype=dtype)
    h = (d + 1) // 2
    coeffs = chebyshev_coefficients(seed, first, count, d, terms, degree)
    for j in range(count):
        f = np.einsum("qmj,jn->qmn", coeffs[j], T)  # [terms, d, n]
        # the sum of separable products as (Khatri-Rao of the first h modes)^T x (of the rest)
        left = np.ones((terms, 1))
        for m in range(h):
            left = (left[:, :, None] * f[:, m, None, :]).reshape(terms, -1)
        right = np.ones((terms, 1))
        for m in range(h, d):
            right = (right[:, :, None] * f[:, m, None, :]).reshape(terms, -1)
        item = (left.T @ right).reshape((n,) * d)
        if noise_std:
            item += noise_std * counter_normals(seed, first + j, item.size).reshape(item.shape)
        out[j] = item
    return out


# ---------------------------------------------------------------------------
# Graded spectrum: a numerical stress stream for tight tolerances
# ---------------------------------------------------------------------------

def graded_stream(seed: int, n1: int = 400, n2: int = 6, N: int = 48, rank: int = 288,
                  decades: float = 6.0, offsets=(0, 112, 50)) -> list:
    """Batches of two-way items [N, n1, n2], float64, one per entry of ``offsets``.

    A fixed random orthonormal basis P of R^{n1} is drawn once per stream. In batch k the
    mode-1 unfolding [n1, N * n2] equals P[:, o_k .. o_k + rank - 1] diag(s) W_k^T, with
    s_i = 10^(-decades * i / (rank - 1)) and W_k random with orthonormal columns, so its
    singular values are exactly s: the Gram spectrum spans 2 * decades decades and the
    eigenvalues below 1e-9 of the largest are many and closely spaced.
    """
    rng = np.random.default_rng([int(seed), 7_000_003])
    P = np.linalg.qr(rng.normal(size=(n1, n1)))[0]
    s = 10.0 ** (-decades * np.arange(rank) / max(rank - 1, 1))
    out = []
    for o in offsets:
        if o + rank > n1:
            raise ValueError("offset + rank exceeds n1")
        W = np.linalg.qr(rng.normal(size=(N * n2, rank)))[0]
        M = (P[:, o:o + rank] * s) @ W.T
        out.append(np.ascontiguousarray(M.reshape(n1, N, n2).transpose(1, 0, 2)))
    return out
