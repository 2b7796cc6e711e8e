"""Seeded synthetic inputs for FCG-NO solves: coefficient fields, right-hand sides, initial
guesses and neural-operator weight blobs.

This module only draws random numbers and lays them out. It holds none of the method's
arithmetic (no stencil, no Krylov step, no Fourier transform of the solver), so both the
CUDA path and the FP64 oracle consume exactly the same arrays.

Grid convention used throughout: an N x N grid of interior nodes of the unit square,
node (p, q) at x1 = (p+1) h, x2 = (q+1) h with h = 1/(N+1); arrays are indexed [q][p]
(p, the x1 index, fastest), i.e. unknown index q*N + p.

Problem families
- ``grf_coefficient``: k = exp(g), g a Gaussian random field with squared-exponential
  covariance sigma^2 exp(-|x-y|^2 / (2 l^2)) on the interior nodes, sampled separably as
  g = sigma * L Z L^T with L the symmetric square root of the 1-D correlation matrix
  (negative eigenvalues clamped to zero).
- ``trig_polynomial``: the paper's random trigonometric polynomial P(N1, N2, alpha)
  (Section 3.2, datasets): g(x) = sum_{m<=N1, n<=N2} c_mn exp(2 pi i (m x1 + n x2)) /
  (1+m+n)^alpha with complex standard-normal c_mn; the garbled "R(c) ~ N(0, I)" is read
  as f = Re g.
- ``poisson_problem`` / ``diffusion_problem``: the paper's two datasets (Section 3.2):
  a = 1, f ~ P(5,5,2) and a ~ P(5,5,2) + 10, f ~ P(5,5,2).
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "ModelDesc",
    "grf_coefficient",
    "gaussian_rhs",
    "make_problem",
    "make_batch",
    "trig_polynomial",
    "poisson_problem",
    "diffusion_problem",
    "xavier_weights",
    "weight_count",
    "weight_offsets",
    "mode_k1_index",
]


@dataclass(frozen=True)
class ModelDesc:
    """Shape of the Fourier neural operator preconditioner.

    width: channel count C of the processor; layers: number of Fourier layers;
    modes: M, giving 2M retained x1-frequencies (0..M-1 and -M..-1) and M retained
    x2-frequencies (0..M-1); proj_width: hidden width of the projection (C_p);
    in_channels: 2 (normalised residual and log k).
    """

    width: int = 32
    layers: int = 4
    modes: int = 12
    proj_width: int = 32
    in_channels: int = 2
    output_scale: int = 0  # 0: output times h^2 rms(r); 1: also divided by k at every grid point

    @property
    def kx(self) -> int:
        return 2 * self.modes

    @property
    def ky(self) -> int:
        return self.modes


def weight_offsets(desc: ModelDesc) -> dict:
    """Offsets (in float32 elements) of every parameter inside the flat weight blob.

    Order and shapes (all row-major):
      lift_w  [C][in_channels]   lift_b [C]
      per layer l: w{l} [C][C] (out, in), b{l} [C],
                   r{l} [2M][M][C][C][2] (kx index, ky, in, out, re/im)
      proj1_w [C_p][C], proj1_b [C_p], proj2_w [C_p], proj2_b [1]
    The kx index j maps to the signed frequency j for j < M and j - 2M for j >= M.
    """
    C, Cp, L, M, ci = desc.width, desc.proj_width, desc.layers, desc.modes, desc.in_channels
    off = {}
    pos = 0

    def put(name, size):
        nonlocal pos
        off[name] = (pos, size)
        pos += size

    put("lift_w", C * ci)
    put("lift_b", C)
    for l in range(L):
        put(f"w{l}", C * C)
        put(f"b{l}", C)
        put(f"r{l}", 2 * M * M * C * C * 2)
    put("proj1_w", Cp * C)
    put("proj1_b", Cp)
    put("proj2_w", Cp)
    put("proj2_b", 1)
    off["_total"] = (pos, 0)
    return off


def weight_count(desc: ModelDesc) -> int:
    return weight_offsets(desc)["_total"][0]


def mode_k1_index(j: int, modes: int) -> int:
    """Signed x1-frequency of kx slot j (0 <= j < 2*modes)."""
    return j if j < modes else j - 2 * modes


def xavier_weights(desc: ModelDesc, seed: int = 0) -> np.ndarray:
    """Xavier-uniform initial weights as one float32 blob (biases zero).

    Every real matrix of shape (out, in) is drawn from U(-a, a) with
    a = sqrt(6 / (in + out)); the spectral weights draw their real and imaginary parts
    separately with fan_in = fan_out = C. Draw order follows the blob order.
    """
    rng = np.random.default_rng(seed)
    C, Cp, L, M, ci = desc.width, desc.proj_width, desc.layers, desc.modes, desc.in_channels
    off = weight_offsets(desc)
    blob = np.zeros(weight_count(desc), dtype=np.float64)

    def xav(shape, fan_in, fan_out):
        a = math.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-a, a, size=shape)

    o, s = off["lift_w"]
    blob[o:o + s] = xav((C, ci), ci, C).ravel()
    for l in range(L):
        o, s = off[f"w{l}"]
        blob[o:o + s] = xav((C, C), C, C).ravel()
        o, s = off[f"r{l}"]
        re = xav((2 * M, M, C, C), C, C)
        im = xav((2 * M, M, C, C), C, C)
        blob[o:o + s] = np.stack([re, im], axis=-1).ravel()
    o, s = off["proj1_w"]
    blob[o:o + s] = xav((Cp, C), C, Cp).ravel()
    o, s = off["proj2_w"]
    blob[o:o + s] = xav((1, Cp), Cp, 1).ravel()
    return blob.astype(np.float32)


@functools.lru_cache(maxsize=16)
def _sqrt_corr_1d(N: int, ell: float) -> np.ndarray:
    """Symmetric square root of the 1-D correlation matrix of the interior nodes (cached: it
    depends on N and ell only; callers must not modify it)."""
    h = 1.0 / (N + 1)
    x = (np.arange(N) + 1) * h
    d = x[:, None] - x[None, :]
    c = np.exp(-(d * d) / (2.0 * ell * ell))
    lam, V = np.linalg.eigh(c)
    lam = np.clip(lam, 0.0, None)
    return (V * np.sqrt(lam)) @ V.T


def grf_coefficient(N: int, rng: np.random.Generator, sigma: float = 1.0, ell: float = 0.1) -> np.ndarray:
    """k = exp(g) on the interior nodes, g ~ GRF(0, sigma^2 exp(-d^2/(2 ell^2))); [N][N] float64."""
    L = _sqrt_corr_1d(N, ell)
    Z = rng.standard_normal((N, N))
    g = sigma * (L @ Z @ L.T)
    return np.exp(g)


def gaussian_rhs(N: int, rng: np.random.Generator) -> np.ndarray:
    """f iid N(0,1) at the interior nodes; [N][N] float64."""
    return rng.standard_normal((N, N))


def make_problem(N: int, seed: int, sigma: float = 1.0, ell: float = 0.1):
    """One diffusion instance: (k, f), both [N][N] float64, from one seed."""
    rng = np.random.default_rng(seed)
    k = grf_coefficient(N, rng, sigma, ell)
    f = gaussian_rhs(N, rng)
    return k, f


def make_batch(N: int, seeds, sigma: float = 1.0, ell: float = 0.1):
    """Stacked instances: k, f of shape [B][N][N] float64 (one seed per instance)."""
    ks, fs = [], []
    for s in seeds:
        k, f = make_problem(N, int(s), sigma, ell)
        ks.append(k)
        fs.append(f)
    return np.ascontiguousarray(np.stack(ks)), np.ascontiguousarray(np.stack(fs))


def trig_polynomial(N: int, rng: np.random.Generator, N1: int = 5, N2: int = 5, alpha: float = 2.0) -> np.ndarray:
    """Random trigonometric polynomial P(N1, N2, alpha) sampled at the interior nodes."""
    h = 1.0 / (N + 1)
    x = (np.arange(N) + 1) * h
    c = rng.standard_normal((N1 + 1, N2 + 1)) + 1j * rng.standard_normal((N1 + 1, N2 + 1))
    m = np.arange(N1 + 1)[:, None]
    n = np.arange(N2 + 1)[None, :]
    c = c / (1.0 + m + n) ** alpha
    e1 = np.exp(2j * np.pi * np.outer(np.arange(N1 + 1), x))   # [m][p]
    e2 = np.exp(2j * np.pi * np.outer(np.arange(N2 + 1), x))   # [n][q]
    g = np.einsum("mn,mp,nq->qp", c, e1, e2)
    return np.real(g)


def poisson_problem(N: int, seed: int):
    """Paper's Poisson dataset: k = 1, f ~ P(5,5,2)."""
    rng = np.random.default_rng(seed)
    return np.ones((N, N)), trig_polynomial(N, rng)


def diffusion_problem(N: int, seed: int):
    """Paper's Diffusion dataset: k ~ P(5,5,2) + 10, f ~ P(5,5,2)."""
    rng = np.random.default_rng(seed)
    k = trig_polynomial(N, rng) + 10.0
    f = trig_polynomial(N, rng)
    return k, f


# ------------------------------------------------------------------------------ datasets by name
DATASETS = ("grf", "poisson", "diffusion")


def dataset_problem(name: str, N: int, seed: int, sigma: float = 1.0, ell: float = 0.1):
    """(k, f) of instance `seed` of a named family: "grf" (k = exp(GRF), f iid N(0,1)),
    "poisson" or "diffusion" (the paper's datasets, Section 3.2)."""
    if name == "grf":
        return make_problem(N, seed, sigma, ell)
    if name == "poisson":
        return poisson_problem(N, seed)
    if name == "diffusion":
        return diffusion_problem(N, seed)
    raise ValueError(f"unknown dataset {name!r}")


def dataset_rhs(name: str, N: int, rng: np.random.Generator) -> np.ndarray:
    """A right-hand side f ~ p_f of the named family (for the random-residual data of
    Section 3.5: f is redrawn per sample, k stays the instance's)."""
    if name == "grf":
        return gaussian_rhs(N, rng)
    if name in ("poisson", "diffusion"):
        return trig_polynomial(N, rng)
    raise ValueError(f"unknown dataset {name!r}")
