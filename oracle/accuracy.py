"""First-pass accuracy metric (paper Section 6.1, Eq. err_metric).

ORACLE -- test infrastructure only (see oracle/__init__.py).

E_2^chi = sqrt( mean over Omega_s of (E_p^chi)^2 ),
E_p^chi = ||chi_M - chi_S|| / sup_{Omega_s} ||chi_S||,
for chi = u (displacement) and chi = sigma^t, the maximum shear stress
(sigma_max - sigma_min)/2 of the principal stresses.
Readings: u is compared at every existing node (vector 2-norm per node);
sigma^t is evaluated at element centroids with the element's own modulus,
and both means are plain averages over the sample points.
"""
from __future__ import annotations

import numpy as np

from .fem import elasticity_matrix, shape_gradients, strain_matrix


def centroid_stress(system, x):
    """Cauchy stress tensors (n_elem x 3 x 3) at voxel centroids for free-DOF vector x."""
    u = system.expand(x)
    mesh = system.mesh
    B = strain_matrix(shape_gradients((0.5, 0.5, 0.5)))
    D = elasticity_matrix(1.0, system.nu)
    ue = u[mesh.conn].reshape(mesh.n_elem, 24)
    eps = ue @ B.T
    Ee = system.E[mesh.elem_ijk[:, 2], mesh.elem_ijk[:, 1], mesh.elem_ijk[:, 0]]
    s = (eps @ D.T) * Ee[:, None]
    S = np.empty((mesh.n_elem, 3, 3))
    S[:, 0, 0], S[:, 1, 1], S[:, 2, 2] = s[:, 0], s[:, 1], s[:, 2]
    S[:, 1, 2] = S[:, 2, 1] = s[:, 3]
    S[:, 0, 2] = S[:, 2, 0] = s[:, 4]
    S[:, 0, 1] = S[:, 1, 0] = s[:, 5]
    return S


def max_shear(S):
    ev = np.linalg.eigvalsh(S)
    return 0.5 * (ev[:, -1] - ev[:, 0])


def e2_errors(system, x_approx, x_exact):
    """(E_2^u, E_2^{sigma^t}) of an approximate solution against the exact one."""
    uM = system.expand(x_approx)
    uS = system.expand(x_exact)
    du = np.linalg.norm(uM - uS, axis=1)
    e_u = np.sqrt(np.mean((du / np.linalg.norm(uS, axis=1).max()) ** 2))
    tM = max_shear(centroid_stress(system, x_approx))
    tS = max_shear(centroid_stress(system, x_exact))
    e_s = np.sqrt(np.mean((np.abs(tM - tS) / np.abs(tS).max()) ** 2))
    return float(e_u), float(e_s)
