"""Coarse preconditioner M_G (paper Section 4.2, Eqs. mg_struct, WQP,
bc_matrix, col_cg, col_pk, col_ek, contract).

ORACLE -- test infrastructure only (see oracle/__init__.py).

* Eq. mg_struct: M_G^{-1} = P_hat (R_hat A_hat P_hat)^{-1} R_hat, R_hat = P_hat^T.
* Eq. WQP: P_hat = W Q P, so column k of P_hat, written in the original DOF
  order, is [basis vectors on grain DOFs ; column k of Q^o on interface DOFs].
* Eq. bc_matrix / col_pk: shape vector p_k^{g} = -(A^g_g)^{-1} Abar^g_{m} e_k
  with Abar^g_m = A^g_c Q^o (Eq. redu_orig); it is nonzero only on grains
  coupled to the interface hosting mortar column k.
* Eq. col_cg: correction vector c^g = (A^g_g)^{-1} b^g; a correction column is
  kept only when b^g is nonzero (Section 4.2 notes it vanishes otherwise, and
  a zero column would make the coarse matrix singular).
* Column order: mortar columns (interface, mortar, component), then the kept
  correction columns in grain order.
* A^o = P_hat^T A_hat P_hat, checked symmetric to 1e-12 (relative), then
  symmetrised and Cholesky-factored (the paper's "direct solver").
Local solves use a sparse LU (SuperLU through scipy) as a library primitive.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class CoarseSpace:
    def __init__(self, system, dec, mortars, keep_corrections=True):
        A = system.A.tocsr()
        b = system.b
        n = system.n_dof
        self.n_m = mortars.n_mortar_cols
        self.grain_lu = []
        cols_rows, cols_cols, cols_vals = [], [], []
        # interface rows: Q^o columns
        for c in range(dec.n_interfaces):
            Qc = mortars.Qo_block(system, dec, c)
            J = dec.iface_dofs[c]
            off = mortars.iface_col_offset[c]
            r, k = np.nonzero(Qc)
            cols_rows.append(J[r])
            cols_cols.append(off + k)
            cols_vals.append(Qc[r, k])
        self.correction_grain = []
        corr_vectors = []
        for g in range(dec.n_grains):
            I = dec.grain_dofs[g]
            if I.size == 0:
                self.grain_lu.append(None)
                continue
            Agg = A[I][:, I].tocsc()
            lu = spla.splu(Agg)
            self.grain_lu.append(lu)
            for c in dec.grain_ifaces[g]:
                J = dec.iface_dofs[c]
                if J.size == 0:
                    continue
                Qc = mortars.Qo_block(system, dec, c)
                Abar = A[I][:, J] @ Qc                      # Abar^g_m restricted to interface c's columns
                P = -lu.solve(np.asarray(Abar))              # Eq. col_pk
                off = mortars.iface_col_offset[c]
                rr, kk = np.nonzero(P)
                cols_rows.append(I[rr])
                cols_cols.append(off + kk)
                cols_vals.append(P[rr, kk])
            bg = b[I]
            if keep_corrections and np.any(bg != 0.0):
                corr_vectors.append((g, I, lu.solve(bg)))   # Eq. col_cg
        for j, (g, I, cg) in enumerate(corr_vectors):
            self.correction_grain.append(g)
            nz = np.flatnonzero(cg)
            cols_rows.append(I[nz])
            cols_cols.append(np.full(nz.size, self.n_m + j))
            cols_vals.append(cg[nz])
        self.n_coarse = self.n_m + len(corr_vectors)
        rows = np.concatenate(cols_rows) if cols_rows else np.zeros(0, np.int64)
        cols = np.concatenate(cols_cols) if cols_cols else np.zeros(0, np.int64)
        vals = np.concatenate(cols_vals) if cols_vals else np.zeros(0)
        self.P_hat = sp.coo_matrix((vals, (rows, cols)), shape=(n, self.n_coarse)).tocsc()
        AP = (A @ self.P_hat).tocsc()
        Ao = (self.P_hat.T.tocsr() @ AP).toarray()
        scale = max(np.abs(Ao).max(), 1e-300)
        self.asymmetry = float(np.abs(Ao - Ao.T).max() / scale)
        if self.asymmetry > 1e-12:
            raise ValueError(f"coarse matrix asymmetric: {self.asymmetry:.3e}")
        self.A_o = 0.5 * (Ao + Ao.T)
        self.chol = sla.cho_factor(self.A_o, lower=True) if self.n_coarse else None

    def apply(self, r):
        """M_G^{-1} r = P_hat (A^o)^{-1} P_hat^T r (Eq. mg_struct)."""
        if self.n_coarse == 0:
            return np.zeros_like(r)
        return self.P_hat @ sla.cho_solve(self.chol, self.P_hat.T @ r)

    def restrict(self, r):
        return self.P_hat.T @ r

    def prolong(self, u):
        return self.P_hat @ u
