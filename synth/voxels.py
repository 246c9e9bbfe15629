"""Seeded voxel workloads shaped like the paper's pore-scale, continuum and
fractured domains (Section 5, Table "settings"): binary porous solids, a
log-normal modulus field, stiffness contrast and thin compliant slits.

Every array is indexed [z][y][x] (x fastest), matching the voxel numbering
v = x + nx*(y + ny*z) used throughout the library.  Moduli are float32, the
type the library's C interface takes, so both consumers see identical values.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Tuple

import numpy as np
from scipy import ndimage

FACES = ("x0", "x1", "y0", "y1", "z0", "z1")


@dataclasses.dataclass
class Problem:
    """A voxel elasticity problem: geometry, material, subdomains and loads."""
    name: str
    mask: np.ndarray            # uint8 [nz, ny, nx], 1 = solid
    E: np.ndarray               # float32 [nz, ny, nx], Young's modulus per voxel
    nu: float                   # Poisson ratio (global)
    grains: Tuple[int, int, int]  # Cartesian subdomain counts (px, py, pz)
    bcs: Dict[str, dict]        # face -> {"fix": (bx,by,bz), "value": (ux,uy,uz), "traction": (tx,ty,tz)}
    n_mortar: int = 4           # maximum mortar nodes per interface
    seed: int = 0

    @property
    def shape(self):
        return self.mask.shape


def _empty_face():
    return {"fix": (False, False, False), "value": (0.0, 0.0, 0.0), "traction": (0.0, 0.0, 0.0)}


def bcs_clamped_traction(traction=(0.0, 0.0, 1.0), clamp_face="z0", load_face="z1"):
    """Clamp every component on `clamp_face`; uniform traction on `load_face`."""
    bcs = {f: _empty_face() for f in FACES}
    bcs[clamp_face] = {"fix": (True, True, True), "value": (0.0, 0.0, 0.0), "traction": (0.0, 0.0, 0.0)}
    bcs[load_face] = {"fix": (False, False, False), "value": (0.0, 0.0, 0.0),
                      "traction": tuple(float(t) for t in traction)}
    return bcs


def bcs_dict_to_arrays(bcs):
    """Face dictionary -> (fix uint8[6,3], value float64[6,3], traction float64[6,3])."""
    fix = np.zeros((6, 3), np.uint8)
    val = np.zeros((6, 3), np.float64)
    tra = np.zeros((6, 3), np.float64)
    for f, face in enumerate(FACES):
        d = bcs.get(face, _empty_face())
        fix[f] = [1 if b else 0 for b in d["fix"]]
        val[f] = d["value"]
        tra[f] = d["traction"]
    return fix, val, tra


def _largest_component_touching_bottom(solid):
    """Keep the largest 6-connected solid component that touches the z=0 face."""
    lab, n = ndimage.label(solid, structure=ndimage.generate_binary_structure(3, 1))
    if n == 0:
        return np.zeros_like(solid, dtype=np.uint8)
    sizes = np.bincount(lab.ravel(), minlength=n + 1)
    bottom = np.unique(lab[0][lab[0] > 0])
    if bottom.size == 0:
        return np.zeros_like(solid, dtype=np.uint8)
    best = bottom[np.argmax(sizes[bottom])]
    return (lab == best).astype(np.uint8)


def _filtered_noise(rng, shape, sigma):
    noise = rng.standard_normal(shape)
    return ndimage.gaussian_filter(noise, sigma=sigma, mode="reflect", truncate=4.0)


def porous_mask(shape, porosity, sigma, rng):
    """Gaussian-filtered white noise thresholded at the porosity quantile.

    Voxels whose filtered value ranks in the lowest `porosity` fraction become
    void (ties broken by a stable sort), then the largest 6-connected solid
    component touching z=0 is kept so that the clamped problem is nonsingular.
    """
    f = _filtered_noise(rng, shape, sigma).ravel()
    order = np.argsort(f, kind="stable")
    n_void = int(round(porosity * f.size))
    solid = np.ones(f.size, dtype=bool)
    solid[order[:n_void]] = False
    return _largest_component_touching_bottom(solid.reshape(shape))


def lognormal_modulus(shape, sigma_corr, rng, mu=0.0, sigma=1.0):
    """E = exp(mu + sigma*g), g a Gaussian-filtered field rescaled to zero mean, unit variance."""
    g = _filtered_noise(rng, shape, sigma_corr)
    g = (g - g.mean()) / g.std()
    return np.exp(mu + sigma * g).astype(np.float32)


def _slits_and_voronoi(shape, rng, n_slits=20, radius=32.0, n_seeds=64, contrast=1e-4, phases=(1.0, 10.0)):
    from scipy.spatial import cKDTree
    nz, ny, nx = shape
    seeds = rng.uniform(0.0, 1.0, size=(n_seeds, 3)) * np.array([nx, ny, nz])
    phase = rng.integers(0, 2, size=n_seeds)
    tree = cKDTree(seeds)
    E = np.empty(nz * ny * nx, np.float64)
    xs, ys = np.arange(nx) + 0.5, np.arange(ny) + 0.5
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    for k in range(nz):  # one z-layer of voxel centres at a time
        pts = np.stack([xx.ravel(), yy.ravel(), np.full(xx.size, k + 0.5)], axis=1)
        _, near = tree.query(pts)
        E[k * ny * nx:(k + 1) * ny * nx] = np.where(phase[near] == 0, phases[0], phases[1])
    E = E.reshape(shape)
    for _ in range(n_slits):
        c = rng.uniform(0.0, 1.0, size=3) * np.array([nx, ny, nz])
        nrm = rng.standard_normal(3)
        nrm /= np.linalg.norm(nrm)
        # only voxel centres within radius + 1 of the centre can lie on the disk: test that box
        lo = np.maximum(np.floor(c - radius - 1).astype(int), 0)
        hi = np.minimum(np.ceil(c + radius + 1).astype(int), [nx, ny, nz])
        zz, yy2, xx2 = np.meshgrid(np.arange(lo[2], hi[2]) + 0.5, np.arange(lo[1], hi[1]) + 0.5,
                                   np.arange(lo[0], hi[0]) + 0.5, indexing="ij")
        rel = np.stack([xx2 - c[0], yy2 - c[1], zz - c[2]], axis=-1)
        dn = rel @ nrm
        dt2 = (rel * rel).sum(axis=-1) - dn * dn
        hit = (np.abs(dn) <= 0.5) & (dt2 <= radius * radius)
        E[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]][hit] *= contrast
    return E.astype(np.float32)


def make_workload(name, seed=0):
    """Build one of the named workloads (see WORKLOADS for the recipes)."""
    rng = np.random.default_rng(seed)
    if name == "cube16":
        shape = (16, 16, 16)
        mask = np.ones(shape, np.uint8)
        E = np.ones(shape, np.float32)
        return Problem(name, mask, E, 0.25, (2, 2, 2), bcs_clamped_traction(), 4, seed)
    if name in ("porous64", "porous32", "porous24", "porous48"):
        n = int(name[len("porous"):])
        shape = (n, n, n)
        mask = porous_mask(shape, 0.3, 2.0, rng)
        E = lognormal_modulus(shape, 2.0, rng)
        p = n // 16
        return Problem(name, mask, E, 0.3, (p, p, p), bcs_clamped_traction(), 4, seed)
    if name == "porous192":
        # the learned warm start's evaluation images: porosity 0.35, the 64^3 recipe's filter, 12^3 grains
        shape = (192, 192, 192)
        mask = porous_mask(shape, 0.35, 2.0, rng)
        E = lognormal_modulus(shape, 2.0, rng)
        return Problem(name, mask, E, 0.3, (12, 12, 12), bcs_clamped_traction(), 4, seed)
    if name == "porous128":
        shape = (128, 128, 128)
        mask = porous_mask(shape, 0.4, 3.0, rng)
        E = lognormal_modulus(shape, 3.0, rng)
        return Problem(name, mask, E, 0.3, (8, 8, 8), bcs_clamped_traction(), 4, seed)
    if name.startswith("fractured"):
        # fractured<n>: the 256^3 recipe at edge n (16^3-voxel grains); smaller edges keep the slit radius and
        # scale the slit and Voronoi seed counts with the volume (at least 3 slits and 8 seeds)
        n = int(name[len("fractured"):])
        shape = (n, n, n)
        frac = (n / 256.0) ** 3
        mask = porous_mask(shape, 0.25, 2.0, rng)
        E = _slits_and_voronoi(shape, rng, n_slits=max(3, int(round(20 * frac))),
                               n_seeds=max(8, int(round(64 * frac))))
        return Problem(name, mask, E, 0.25, (n // 16,) * 3, bcs_clamped_traction(), 2, seed)
    if name.startswith("tiny"):
        # tiny<n>: porous n^3 block with 2x2x2 subdomains, small enough for dense checks
        n = int(name[4:])
        shape = (n, n, n)
        mask = porous_mask(shape, 0.2, 1.0, rng)
        E = lognormal_modulus(shape, 1.0, rng)
        return Problem(name, mask, E, 0.3, (2, 2, 2), bcs_clamped_traction(), 2, seed)
    raise KeyError(name)


WORKLOADS = {
    "cube16": "16^3 all-solid block, E=1, nu=0.25, 2x2x2 subdomains, z=0 clamped, unit +z traction on z=16",
    "porous64": "64^3 porous block: white noise -> Gaussian sigma=2 -> porosity 0.3 -> largest 6-connected "
                "component touching z=0; log-normal E (mu=0, sigma=1, same filter); nu=0.3; 4x4x4 subdomains",
    "porous128": "128^3 porous block, porosity 0.4, sigma=3, log-normal E, nu=0.3, 8x8x8 subdomains",
    "porous192": "192^3 porous block, porosity 0.35, sigma=2, log-normal E, nu=0.3, 12x12x12 subdomains",
    "fractured256": "256^3 porous block (porosity 0.25, sigma=2), 64-seed Voronoi two-phase E in {1,10}, "
                    "20 planar 1-voxel slits of radius 32 with E x 1e-4, nu=0.25, 16x16x16 subdomains",
}
