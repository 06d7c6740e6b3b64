"""Seeded synthetic microstructures for the periodic unit-cell problem.

This module only produces inputs: per-voxel Lame fields lambda(x), mu(x) on an
n3 x n2 x n1 grid (C order, x1 fastest) and load cases. It contains none of the
solver's arithmetic, so both the CUDA path and the FP64 oracle take their inputs
from here.

Geometries follow the paper's matrix-inclusion benchmark (Sec. 2.1 phase field,
eq. FiePhaIncMat / DenVolIncMat; Sec. 6 cubic inclusion with
f(x) = 1 + nu(x1) nu(x2) nu(x3) (chi - 1)), plus the random spherical inclusions
and lognormal perturbations used for the larger synthetic workloads.

Sampling positions: trapezoidal discretization (TD) samples at the nodes
x_i = (i - 1) h, i = 1..n (0-based: i h); piecewise-constant discretization (PCD)
samples at the cell centres x_i^c = (i - 1/2) h (0-based: (i + 1/2) h).
"""
from __future__ import annotations

import numpy as np

VOIGT_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def lame(E, nu):
    """Lame constants (lambda, mu) of an isotropic phase from Young's modulus and Poisson's ratio."""
    E = np.asarray(E, dtype=np.float64)
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def _sample_coords(n, offset):
    return np.arange(n, dtype=np.float64) + offset


def cube_indicator(n, edge):
    """Sharp cubic inclusion defined by voxel index: start <= i_r < start + edge on every axis.

    For edge = n/2 this is n/4 <= i_r < 3n/4; no sample lies on the interface.
    """
    n1, n2, n3 = (n, n, n) if np.isscalar(n) else n
    ind = []
    for nr in (n1, n2, n3):
        a = (nr - edge) // 2
        i = np.arange(nr)
        ind.append(((i >= a) & (i < a + edge)).astype(np.float64))
    return ind[2][:, None, None] * ind[1][None, :, None] * ind[0][None, None, :]


def phase_profile(n, c_l, c_r, eps, offset):
    """1D inclusion density nu_eps(x) = phi(x; c_l) - phi(x; c_r), phi = 1/2 + 1/2 tanh((x - c)/eps).

    eps = 0 gives the sharp limit with theta(0) = 1/2 (eq. FiePhaIncMat, DenVolIncMat).
    """
    x = _sample_coords(n, offset)
    if eps == 0.0:
        def th(d):
            return np.where(d > 0, 1.0, np.where(d < 0, 0.0, 0.5))
        return th(x - c_l) - th(x - c_r)
    return (0.5 + 0.5 * np.tanh((x - c_l) / eps)) - (0.5 + 0.5 * np.tanh((x - c_r) / eps))


def cube_density(n, edge, eps, sampling="TD"):
    """Product density f0(x) = nu(x1) nu(x2) nu(x3) of a centred cube [a, a+edge)^3 in cell [0, n)^3."""
    offset = 0.0 if sampling == "TD" else 0.5
    a = (n - edge) / 2.0
    nu = phase_profile(n, a, a + edge, eps, offset)
    return nu[:, None, None] * nu[None, :, None] * nu[None, None, :]


def two_phase_fields(indicator, E_m, E_i, nu_m=0.3, nu_i=0.3, mixing="sharp"):
    """Per-voxel (lambda, mu) from an inclusion density in [0, 1].

    mixing = "sharp": density must be 0/1 (or 1/2 on an interface) and moduli are mixed linearly.
    mixing = "log":   log E(x) = log E_m + f(x) log(E_i / E_m), with nu fixed (smooth tanh interface).
    mixing = "paper": lambda, mu proportional to 1 + f(x) (chi - 1) (Sec. 6 mixing of the Lame fields).
    """
    f = np.asarray(indicator, dtype=np.float64)
    lm, mm = lame(E_m, nu_m)
    li, mi = lame(E_i, nu_i)
    if mixing == "log":
        if nu_m != nu_i:
            raise ValueError("log mixing assumes one Poisson ratio")
        E = np.exp(np.log(E_m) + f * np.log(E_i / E_m))
        return lame(E, nu_m)
    if mixing in ("sharp", "paper"):
        return lm + f * (li - lm), mm + f * (mi - mm)
    raise ValueError(mixing)


def sharp_cube(n, edge, E_m=1.0, E_i=10.0, nu=0.3):
    """Config: sharp cube of edge `edge` voxels (by voxel index), isotropic phases."""
    return two_phase_fields(cube_indicator(n, edge), E_m, E_i, nu, nu)


def smooth_cube(n, edge, contrast, width=2.0, E_m=1.0, nu=0.3, sampling="TD"):
    """Config: centred cube with a tanh interface of half-width `width` voxels in log-moduli."""
    f = cube_density(n, edge, width, sampling)
    return two_phase_fields(f, E_m, E_m * contrast, nu, nu, mixing="log")


def random_spheres_indicator(n, vf, rmin, rmax, seed, max_tries=200000):
    """Random sequential addition of non-overlapping periodic spheres until the voxel fraction >= vf.

    Radii are uniform in [rmin, rmax] voxels, centres uniform in the cell (numpy PCG64 with `seed`).
    Two spheres may not overlap under the periodic distance (centre distance >= r1 + r2).
    A voxel belongs to a sphere when its centre (i + 1/2) lies within the radius.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n1, n2, n3 = (n, n, n) if np.isscalar(n) else n
    dims = np.array([n1, n2, n3], dtype=np.float64)
    ind = np.zeros((n3, n2, n1), dtype=bool)
    centres = np.zeros((0, 3))
    radii = np.zeros(0)
    tries = 0
    filled = 0
    target = vf * ind.size
    while filled < target and tries < max_tries:
        tries += 1
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(0.0, 1.0, size=3) * dims
        if radii.size:
            d = np.abs(centres - c)
            d = np.minimum(d, dims - d)
            if np.any(np.sqrt((d * d).sum(axis=1)) < r + radii):
                continue
        centres = np.vstack([centres, c])
        radii = np.append(radii, r)
        # voxel-centre test within the sphere's periodic bounding box
        sl = []
        for ax in range(3):
            lo = int(np.floor(c[ax] - r - 1))
            hi = int(np.ceil(c[ax] + r + 1))
            sl.append(np.arange(lo, hi))
        ix, iy, iz = sl
        dx = (ix + 0.5 - c[0])
        dy = (iy + 0.5 - c[1])
        dz = (iz + 0.5 - c[2])
        inside = (dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2) <= r * r
        zz, yy, xx = np.nonzero(inside)
        sel = (iz[zz] % n3, iy[yy] % n2, ix[xx] % n1)
        filled += int(np.count_nonzero(~ind[sel]))
        ind[sel] = True
    return ind.astype(np.float64), list(zip(centres, radii))


def random_spheres(n, vf=0.25, rmin=6.0, rmax=16.0, contrast=100.0, seed=0, E_m=1.0, nu=0.3):
    """Config: random non-overlapping voxelised spheres, inclusion E = contrast * E_m, nu = 0.3."""
    ind, _ = random_spheres_indicator(n, vf, rmin, rmax, seed)
    return two_phase_fields(ind, E_m, E_m * contrast, nu, nu)


def lognormal_perturb(lam, mu, sigma=0.1, seed=0):
    """Multiply lambda and mu by independent seeded lognormal factors exp(sigma z), z ~ N(0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z1 = rng.standard_normal(np.shape(lam))
    z2 = rng.standard_normal(np.shape(mu))
    return lam * np.exp(sigma * z1), mu * np.exp(sigma * z2)


def laminate(n1, n2, n3, lam_profile, mu_profile):
    """Layered medium whose moduli vary along x1 only (lam_profile, mu_profile have length n1)."""
    lam = np.broadcast_to(np.asarray(lam_profile, np.float64)[None, None, :], (n3, n2, n1)).copy()
    mu = np.broadcast_to(np.asarray(mu_profile, np.float64)[None, None, :], (n3, n2, n1)).copy()
    return lam, mu


def random_laminate(n1, n2, n3, seed=0, lo=0.5, hi=20.0):
    """Laminate with seeded log-uniform moduli per layer (x1 index)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    E = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n1))
    nu = rng.uniform(0.15, 0.4, size=n1)
    lam, mu = lame(E, nu)
    return laminate(n1, n2, n3, lam, mu)


def random_field(n1, n2, n3, seed=0, lo=0.5, hi=5.0):
    """Seeded voxelwise-random moduli (white noise), for small parity cases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    E = np.exp(rng.uniform(np.log(lo), np.log(hi), size=(n3, n2, n1)))
    nu = rng.uniform(0.1, 0.4, size=(n3, n2, n1))
    return lame(E, nu)


def batch_specs(count=32, seed=0, sizes=(64, 96, 128)):
    """Specs of the batched homogenization workload: per item n, volume fraction, contrast, seed.

    n is drawn from `sizes`, the volume fraction uniform in [0.1, 0.3], the contrast
    log-uniform in [1e-2, 1e3]; sphere radii U[6, 16] are scaled by n / 128.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(count):
        n = int(rng.choice(sizes))
        vf = float(rng.uniform(0.1, 0.3))
        contrast = float(np.exp(rng.uniform(np.log(1e-2), np.log(1e3))))
        out.append(dict(n=n, vf=vf, contrast=contrast, seed=int(1000 + s),
                        rmin=6.0 * n / 128.0, rmax=16.0 * n / 128.0))
    return out


def batch_item(spec):
    """Fields of one batched-workload item from `batch_specs`."""
    return random_spheres(spec["n"], spec["vf"], spec["rmin"], spec["rmax"], spec["contrast"], spec["seed"])


def voigt_unit_strain(J):
    """Macroscopic strain tensor components (11,22,33,23,13,12) of Voigt unit load J (shear = 1/2)."""
    E = np.zeros(6)
    E[J] = 1.0 if J < 3 else 0.5
    return E
