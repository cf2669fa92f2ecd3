"""Seeded synthetic inputs shared by the tests, the benchmark and users.

This module holds no arithmetic of the recombination method: it only draws
fields with the shapes and statistics of the paper's workloads (a
(24 kpc)^3 periodic box, Sec. II.C; Batchelor-like k^2 density spectra,
Eq. Batchelor) and fixes the redshift grid and the Ly-alpha emission profile
table.  The MHD snapshots of the paper are not available; these Gaussian
random fields stand in for them.

Recipe
  density    ln Delta = sigma g - ln <exp(sigma g)>, g a unit-variance Gaussian
             random field with P(k) ~ k^2 for 0 < |k| <= k_max (integer
             wavenumbers of the box), so <Delta> = 1 exactly.
  velocity   three independent fields of the same spectral shape, each
             normalised to an rms of sigma_v km/s (0 means no flow).
  redshifts  n_steps + 1 nodes uniform in ln(1+z).
  profile    inverse CDF of the thermal Doppler profile exp(-x^2)/sqrt(pi)
             (x in Doppler units, Appendix A) at the M quantiles (k+1/2)/M.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = ["gaussian_field", "density_field", "velocity_field", "z_schedule", "doppler_quantiles",
           "BoxConfig", "CONFIGS", "make_box", "pack_vel4"]


def _k_magnitude(n: int) -> np.ndarray:
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kz = np.fft.rfftfreq(n, d=1.0 / n)
    kx, ky, kzz = np.meshgrid(k1, k1, kz, indexing="ij")
    return np.sqrt(kx * kx + ky * ky + kzz * kzz)


def gaussian_field(n: int, seed: int, stream: int = 0, k_max: float | None = None,
                   spectral_index: float = 2.0) -> np.ndarray:
    """Unit-variance, zero-mean Gaussian random field on an n^3 periodic grid.

    Power spectrum P(k) ~ k^spectral_index for 0 < |k| <= k_max (default n/2).
    Returned as float64 with shape (n, n, n), index order (z, y, x).
    """
    rng = np.random.default_rng([int(seed), int(stream), n])
    white = rng.standard_normal((n, n, n))
    fk = np.fft.rfftn(white)
    k = _k_magnitude(n)
    kmax = n / 2 if k_max is None else float(k_max)
    amp = np.where((k > 0) & (k <= kmax), k ** (spectral_index / 2.0), 0.0)
    g = np.fft.irfftn(fk * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


def density_field(n: int, sigma_lnrho: float, seed: int, k_max: float | None = None) -> np.ndarray:
    """Log-normal overdensity Delta = rho_b/<rho_b> with mean exactly one."""
    g = gaussian_field(n, seed, stream=1, k_max=k_max)
    e = np.exp(sigma_lnrho * g)
    return e / e.mean()


def velocity_field(n: int, sigma_v: float, seed: int, k_max: float | None = None) -> np.ndarray:
    """Peculiar velocity [n^3, 3] in km/s, components (Ux, Uy, Uz)."""
    if sigma_v == 0:
        return np.zeros((n * n * n, 3))
    comps = [gaussian_field(n, seed, stream=2 + a, k_max=k_max).ravel() * sigma_v for a in range(3)]
    return np.stack(comps, axis=1)


def z_schedule(z_start: float, z_end: float, n_steps: int) -> np.ndarray:
    """n_steps + 1 node redshifts, uniform in ln(1+z), from z_start to z_end."""
    y = np.linspace(np.log1p(z_start), np.log1p(z_end), n_steps + 1)
    z = np.expm1(y)
    z[0], z[-1] = z_start, z_end
    return z


def doppler_quantiles(M: int = 4097) -> np.ndarray:
    """Emission-frequency table: x_k with CDF(x_k) = (k + 1/2)/M for exp(-x^2)/sqrt(pi)."""
    from scipy.special import erfinv
    q = (np.arange(M) + 0.5) / M
    return erfinv(2.0 * q - 1.0)


@dataclasses.dataclass(frozen=True)
class BoxConfig:
    name: str
    n: int
    sigma_lnrho: float
    sigma_v: float
    n_packets: int
    n_steps: int
    z_start: float
    z_end: float
    k_max: float | None = None
    precision: str = "mixed"


# The five workloads: FP64 32^3; 128^3 mixed; 256^3 (adjoint); batched boxes; 512^3.
CONFIGS = {
    "box32_fp64": BoxConfig("box32_fp64", 32, 0.3, 0.0, 100_000, 50, 1600.0, 900.0, None, "fp64"),
    "box128_mixed": BoxConfig("box128_mixed", 128, 1.0, 1.0, 10_000_000, 200, 1600.0, 700.0, 32.0, "mixed"),
    "box256": BoxConfig("box256", 256, 0.8, 1.0, 100_000_000, 400, 1800.0, 600.0, None, "mixed"),
    "box512_mixed": BoxConfig("box512_mixed", 512, 1.2, 2.0, 1_000_000_000, 600, 1800.0, 500.0, None, "mixed"),
}


def batched_configs(seed: int = 7, n_boxes: int = 64):
    """Batched workload: box sides uniform in {32,48,64,96,128}, sigma_lnrho in
    [0.1, 1.5], 1e6 packets per 32^3 scaled by volume."""
    rng = np.random.default_rng([seed, 99])
    sides = rng.choice([32, 48, 64, 96, 128], size=n_boxes)
    sig = rng.uniform(0.1, 1.5, size=n_boxes)
    return [BoxConfig(f"batch{i}", int(s), float(g), 1.0, int(round(1e6 * (s / 32) ** 3)), 200, 1600.0, 700.0,
                      None, "mixed") for i, (s, g) in enumerate(zip(sides, sig))]


def make_box(cfg: BoxConfig, seed: int = 1):
    """(delta [n^3], U [n^3, 3] km/s) for a workload, float64."""
    delta = density_field(cfg.n, cfg.sigma_lnrho, seed, cfg.k_max).ravel()
    U = velocity_field(cfg.n, cfg.sigma_v, seed, cfg.k_max)
    return delta, U


def pack_vel4(U: np.ndarray, dtype=np.float32) -> np.ndarray:
    """Interleave (Ux, Uy, Uz, 0) per cell: the [n^3, 4] layout of the velocity buffer."""
    U = np.asarray(U).reshape(-1, 3)
    out = np.zeros((U.shape[0], 4), dtype=dtype)
    out[:, :3] = U
    return out
