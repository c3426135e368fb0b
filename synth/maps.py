"""Synthetic patient maps on a 3-D lattice.

The paper initialises its lattice from per-voxel MRI estimates: a cell
density (v_c) and perfusion (K_trans, v_p), Sections 2.1 and 3.4.  Those
patient data are not available, so seeded Gaussian random fields stand in
for them.  The means are the paper's initial densities for its runtime study
(cell density 0.4, vessel density 0.12, Section 3.2).

Recipe (all free parameters of this stand-in, not values from the paper):

* two independent white-noise fields z1, z2 ~ N(0, 1) per site, drawn from
  numpy's PCG64 generator seeded with ``seed`` (the paper also uses a PCG
  generator, Section 2.6);
* each smoothed by a periodic Gaussian filter of standard deviation
  ``corr_len`` sites (applied in Fourier space), then renormalised to zero
  mean and unit variance;
* p_cell   = clip(cell_mean + cell_sd * z1, 0, 1)
* perf     = exp(perf_sigma * z2 - perf_sigma**2 / 2)        (lognormal, mean 1)
* p_vessel = 1 - exp(-lambda0 * perf), lambda0 = -ln(1 - vessel_mean)
  (the probability that a Poisson count with intensity lambda0 * perf is >= 1,
  so a site with perf = 1 holds a vessel with probability vessel_mean).

All maps are float32 arrays of shape (nz, ny, nx), C-contiguous, so the
linear site index is x + nx * (y + ny * z).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class MapSet:
    """The three per-site input maps, float32, shape (nz, ny, nx)."""

    p_cell: np.ndarray
    perf: np.ndarray
    p_vessel: np.ndarray

    @property
    def shape(self):
        return self.p_cell.shape


def gaussian_random_field(shape, corr_len: float, rng: np.random.Generator) -> np.ndarray:
    """Zero-mean, unit-variance periodic Gaussian random field (float64).

    White noise is multiplied in Fourier space by the transfer function of a
    Gaussian kernel with standard deviation ``corr_len`` (in sites).
    """
    import scipy.fft as sfft

    white = rng.standard_normal(size=shape, dtype=np.float64)
    if corr_len <= 0:
        field = white
    else:
        spec = sfft.rfftn(white.astype(np.float32), workers=-1)
        gain = None
        # separable Gaussian transfer function exp(-2 pi^2 sigma^2 f^2)
        for axis, n in enumerate(shape):
            if axis == len(shape) - 1:
                f = np.fft.rfftfreq(n)
            else:
                f = np.fft.fftfreq(n)
            g = np.exp(-2.0 * math.pi ** 2 * corr_len ** 2 * f ** 2).astype(np.float32)
            view = [1] * len(shape)
            view[axis] = g.shape[0]
            g = g.reshape(view)
            gain = g if gain is None else gain * g
        spec *= gain
        field = sfft.irfftn(spec, s=shape, workers=-1).astype(np.float64)
    field -= field.mean()
    sd = field.std()
    if sd > 0:
        field /= sd
    return field


def make_maps(nx: int, ny: int, nz: int, corr_len: float, seed: int,
              cell_mean: float = 0.4, cell_sd: float = 0.2,
              vessel_mean: float = 0.12, perf_sigma: float = 0.5) -> MapSet:
    """Build p_cell, perf and p_vessel for an nx x ny x nz lattice."""
    shape = (nz, ny, nx)
    rng = np.random.default_rng(seed)
    z1 = gaussian_random_field(shape, corr_len, rng)
    z2 = gaussian_random_field(shape, corr_len, rng)
    p_cell = np.clip(cell_mean + cell_sd * z1, 0.0, 1.0)
    perf = np.exp(perf_sigma * z2 - 0.5 * perf_sigma ** 2)
    lam0 = -math.log(1.0 - vessel_mean)
    p_vessel = -np.expm1(-lam0 * perf)
    return MapSet(np.ascontiguousarray(p_cell, dtype=np.float32),
                  np.ascontiguousarray(perf, dtype=np.float32),
                  np.ascontiguousarray(p_vessel, dtype=np.float32))


def replicate_sizes(n_replicates: int, choices=(64, 96, 128, 192), seed: int = 7):
    """Edge lengths for a batch of cubic replicates of uneven size.

    Drawn uniformly from ``choices`` with numpy's PCG64 generator.
    """
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(choices), size=n_replicates)
    return [int(choices[i]) for i in idx]


def biopsy_maps(vox_y: int = 2, vox_x: int = 10, vox_edge: int = 100, seed: int = 0) -> MapSet:
    """Piecewise-constant maps of a 2-D digital biopsy: vox_y x vox_x MRI
    voxels of vox_edge x vox_edge sites each (nz = 1), the layout of the
    paper's biopsy cross-section (Section 3.4: 2 x 10 voxels of 100 x 100
    grid points, the first half of each row in the poorly perfused tumour
    core, the second half at the better perfused edge).

    Per voxel, drawn with numpy's PCG64 generator seeded with ``seed`` (free
    parameters of this stand-in; the paper's per-voxel Tofts estimates are
    patient data):
      core: perf ~ U(0.1, 0.5), vessel fraction ~ U(0.005, 0.02), cell density ~ U(0.5, 0.8)
      edge: perf ~ U(1.0, 2.0), vessel fraction ~ U(0.03, 0.08), cell density ~ U(0.3, 0.6)
    The lattice seeding then places vessels and cells at random inside each
    voxel with those probabilities.
    """
    rng = np.random.default_rng(seed)
    shape = (1, vox_y * vox_edge, vox_x * vox_edge)
    p_cell = np.empty(shape, dtype=np.float32)
    perf = np.empty(shape, dtype=np.float32)
    p_vessel = np.empty(shape, dtype=np.float32)
    for vy in range(vox_y):
        for vx in range(vox_x):
            edge = vx >= vox_x // 2
            lo_hi = ((1.0, 2.0), (0.03, 0.08), (0.3, 0.6)) if edge else ((0.1, 0.5), (0.005, 0.02), (0.5, 0.8))
            pf, pv, pc = (rng.uniform(a, b) for a, b in lo_hi)
            sl = (0, slice(vy * vox_edge, (vy + 1) * vox_edge), slice(vx * vox_edge, (vx + 1) * vox_edge))
            perf[sl], p_vessel[sl], p_cell[sl] = pf, pv, pc
    return MapSet(p_cell, perf, p_vessel)
