"""Brute-force assembly and application of the unfitted DG operator (oracle; test infrastructure).

Bilinear form (paper Sec. 2.1, Eq. bilinear_cg and Eq. bilinear_dg), with a per-cell diffusion coefficient kappa that
multiplies every term linearly (kappa = 1 gives the paper's form exactly):

  a(v, u) = sum_K kappa_K int_{K cap Omega} grad v . grad u                         (Poisson)
          + sum_{K cut} kappa_K int_{Gamma cap K} [ -d_n v u - v d_n u + (tau/h) v u ]  (Nitsche)
          + sum_F int_{F cap Omega} [ -{kappa d_n v}[u] - [v]{kappa d_n u}
                                      + (sigma/h) {kappa} [v][u] ]                  (SIPG)
          + sum_{F in F_G} sum_{j=1..J} gamma_j {kappa} int_F [d_n^j v][d_n^j u]     (ghost penalty)

with [w] = w^- - w^+, {w} = (w^- + w^+) / 2 (Eq. bilinear_dg), n = +e_axis on an interior face from the
lower cell K^- to the upper cell K^+, n = grad phi / |grad phi| on Gamma (outward), h the
background cell size, gamma_j = gp_gamma * h^(2j-1) / (j!)^2, and F_G the interior faces between
two active cells at least one of which is cut.  The ghost penalty is the face-based variant
(the paper's Sec. 2.2 names it and cites Burman 2010); its jump orders 1..J act on the full face.

Quadrature (Sec. 2.3): inside cells and full faces use the tensor Gauss rule with n = p + 1 points
per direction (exact for every integrand above on a Cartesian cell); cut cells and cut faces use
the dimension-reduction rules of ``saye``; the ghost penalty always uses the full-face Gauss rule.

Every basis function is evaluated naively at every point as the full product
phi_l(x) = prod_a phi_{l_a}(xi_a) (Eq. naive_evaluation, Sec. 3.2); local matrices are sums over points of outer
products; nothing is sum-factorised.
"""
import math

import numpy as np
import scipy.sparse as sp

from . import basis, mesh, saye


class Oracle:
    """discretization = "dg": the SIPG operator of Eq. bilinear_dg; "cg": the continuous
    operator of Eq. bilinear_cg (Poisson + Nitsche) with the face ghost penalty, on the
    continuous Q_p space whose nodes are the Gauss-Lobatto lattice points of the active cells."""

    def __init__(self, prob, discretization="dg"):
        if discretization not in ("dg", "cg"):
            raise ValueError("discretization must be 'dg' or 'cg'")
        self.discretization = discretization
        self.prob = prob
        self.mesh = mesh.Mesh(prob)
        self.n = prob.n
        self.nodes = basis.gauss_lobatto_nodes(self.n)
        self.ndof = prob.dofs_per_cell
        d = prob.dim
        # multi-index of every local DoF, l = i + n j + n^2 k
        self.lidx = np.array([[(l // self.n ** a) % self.n for a in range(d)]
                              for l in range(self.ndof)])
        self._cell_q = {}
        self._face_q = {}

    # ----------------------------------------------------------------- quadrature
    def cell_quadrature(self, e):
        """(volume points, weights), (surface points, weights, normals) of active cell e."""
        if e not in self._cell_q:
            prob = self.prob
            lo, hi = mesh.cell_box(prob, self.mesh.index_of(e))
            if self.mesh.active_type[e] == mesh.INSIDE:
                vol = saye.tensor_gauss(lo, hi, self.n)
                surf = []
            else:
                vol, surf = saye.cell_rules(prob, lo, hi)
            vx = np.array([p for p, _ in vol]).reshape(-1, prob.dim)
            vw = np.array([w for _, w in vol])
            sx = np.array([p for p, _, _ in surf]).reshape(-1, prob.dim)
            sw = np.array([w for _, w, _ in surf])
            sn = np.array([nn for _, _, nn in surf]).reshape(-1, prob.dim)
            self._cell_q[e] = (vx, vw, sx, sw, sn)
        return self._cell_q[e]

    def face_quadrature(self, e_minus, axis, full=False):
        """Points and weights on F cap Omega (full=False) or on the whole face F (full=True)."""
        key = (e_minus, axis, full)
        if key not in self._face_q:
            lo, hi = self.mesh.face_box(e_minus, axis)
            ftype = self.mesh.face_type(e_minus, axis)
            if full or ftype == mesh.FACE_FULL:
                # tensor Gauss rule on the (d-1)-dimensional face
                sub = saye.tensor_gauss(saye._drop(lo, axis), saye._drop(hi, axis), self.n)
                pts = [(saye._insert(x, axis, lo[axis]), w) for (x, w) in sub]
            elif ftype == mesh.FACE_EMPTY:
                pts = []
            else:
                pts = saye.face_rule(self.prob, lo, hi, axis)
            fx = np.array([p for p, _ in pts]).reshape(-1, self.prob.dim)
            fw = np.array([w for _, w in pts])
            self._face_q[key] = (fx, fw)
        return self._face_q[key]

    # ----------------------------------------------------------------- basis at points
    def basis_at(self, e, X, deriv_axis=None, order=0, fixed=None):
        """B[q, l] = d^order/dx_axis^order phi_l(X[q]) for the shape functions of cell e.

        fixed = (axis, xi) pins the reference coordinate of `axis` (points on a face).
        """
        prob = self.prob
        lo, _ = mesh.cell_box(prob, self.mesh.index_of(e))
        h = prob.h
        B = np.ones((len(X), self.ndof))
        for a in range(prob.dim):
            xi = (X[:, a] - lo[a]) / h
            if fixed is not None and fixed[0] == a:
                xi = np.full(len(X), float(fixed[1]))
            o = order if a == deriv_axis else 0
            V = basis.lagrange_eval(self.nodes, xi, o) / h ** o
            B = B * V[:, self.lidx[:, a]]
        return B

    def grad_at(self, e, X, fixed=None):
        return [self.basis_at(e, X, a, 1, fixed) for a in range(self.prob.dim)]

    # ----------------------------------------------------------------- local matrices
    def cell_matrix(self, e, kappa_scale=True):
        """Poisson (and, on cut cells, Nitsche) matrix of cell e, rows = test functions."""
        prob = self.prob
        vx, vw, sx, sw, sn = self.cell_quadrature(e)
        kap = self.mesh.kappa[e] if kappa_scale else 1.0
        A = np.zeros((self.ndof, self.ndof))
        if len(vw):
            for G in self.grad_at(e, vx):
                A += G.T @ (vw[:, None] * G)
        if len(sw):
            V = self.basis_at(e, sx)
            G = self.grad_at(e, sx)
            Dn = sum(sn[:, a:a + 1] * G[a] for a in range(prob.dim))
            tau = prob.nitsche_gamma / prob.h
            A += -Dn.T @ (sw[:, None] * V) - V.T @ (sw[:, None] * Dn) + tau * (V.T @ (sw[:, None] * V))
        return kap * A

    def _face_setup(self, e_minus, axis):
        m = self.mesh
        e_plus = m.neighbor(e_minus, axis, 1)
        kap = (m.kappa[e_minus], m.kappa[e_plus])
        return (e_minus, e_plus), kap, 0.5 * (kap[0] + kap[1])

    def sipg_blocks(self, e_minus, axis):
        """Blocks {(s, t): A_st} of the SIPG form on F cap Omega for the face between e_minus
        (side 0 = '-') and its upper neighbour (side 1 = '+'); rows = test functions of side s.

        [phi^s] = sgn_s phi^s with sgn = (+1, -1); {kappa d_n phi^s} = kappa_s d_n phi^s / 2."""
        prob = self.prob
        cells, kap, kavg = self._face_setup(e_minus, axis)
        sgn = (1.0, -1.0)
        xi_face = (1.0, 0.0)
        blocks = {(s, t): np.zeros((self.ndof, self.ndof)) for s in range(2) for t in range(2)}
        fx, fw = self.face_quadrature(e_minus, axis)
        if len(fw):
            V = [self.basis_at(cells[s], fx, fixed=(axis, xi_face[s])) for s in range(2)]
            D = [self.basis_at(cells[s], fx, axis, 1, fixed=(axis, xi_face[s])) for s in range(2)]
            sig = prob.sipg_gamma / prob.h
            Wt = fw[:, None]
            for s in range(2):
                for t in range(2):
                    blocks[(s, t)] += (-0.5 * kap[s] * sgn[t] * (D[s].T @ (Wt * V[t]))
                                       - 0.5 * kap[t] * sgn[s] * (V[s].T @ (Wt * D[t]))
                                       + sig * kavg * sgn[s] * sgn[t] * (V[s].T @ (Wt * V[t])))
        return blocks

    def volume_gp_patches(self):
        """Faces (e_minus, axis) of the volume ghost penalty's patches, stable-neighbour strategy
        (Sec. 2.2): every cut cell is paired across one face with its active face neighbour of
        largest physical volume fraction |K cap Omega| / h^d (inside cells: 1; fractions compared
        after rounding to 12 decimals; the first face in the order axis 0 lower, axis 0 upper,
        axis 1 lower, ... wins ties); a pair chosen from both sides is one patch."""
        if getattr(self, "_patches", None) is None:
            m = self.mesh
            d = self.prob.dim
            frac = np.ones(m.n_active)
            for e in range(m.n_active):
                if m.active_type[e] == mesh.CUT:
                    frac[e] = self.cell_quadrature(e)[1].sum() / self.prob.h ** d
            key = np.floor(frac * 1e12 + 0.5)
            patches = set()
            for e in range(m.n_active):
                if m.active_type[e] != mesh.CUT:
                    continue
                best = None
                for axis in range(d):
                    for side in range(2):
                        nb = m.neighbor(e, axis, side)
                        if nb >= 0 and (best is None or key[nb] > key[best[0]]):
                            best = (nb, axis, side)
                if best is not None:
                    nb, axis, side = best
                    patches.add((e if side == 1 else nb, axis))
            self._patches = patches
        return self._patches

    def volume_gp_blocks(self, e_minus, axis):
        """Blocks of the volume ghost penalty tau_v / h^2 {kappa} int_P [v]_P [u]_P on the patch
        P = K- cup K+ (Sec. 2.2, Eq. volume_based_gp): on each cell of the patch [u]_P is the own
        polynomial minus the other cell's polynomial extended to it (Sec. 3.3), integrated with the
        tensor Gauss rule of the full cell."""
        prob = self.prob
        cells, kap, kavg = self._face_setup(e_minus, axis)
        blocks = {(s, t): np.zeros((self.ndof, self.ndof)) for s in range(2) for t in range(2)}
        c = prob.gp_tau / prob.h ** 2 * kavg
        for owner in range(2):
            lo, hi = mesh.cell_box(prob, self.mesh.index_of(cells[owner]))
            pts = saye.tensor_gauss(lo, hi, self.n)
            X = np.array([x for x, _ in pts])
            w = np.array([wt for _, wt in pts])
            V = [self.basis_at(cells[s], X) for s in range(2)]  # extrapolated for s != owner
            sg = [1.0 if s == owner else -1.0 for s in range(2)]
            for s in range(2):
                for t in range(2):
                    blocks[(s, t)] += c * sg[s] * sg[t] * (V[s].T @ (w[:, None] * V[t]))
        return blocks

    def gp_blocks(self, e_minus, axis):
        """Blocks of the ghost penalty of one interior face: face-based, sum_j gamma_j {kappa}
        int_F [d_n^j v][d_n^j u] on the full face (zero unless one of the two cells is cut); or
        volume-based on the patches of volume_gp_patches."""
        prob = self.prob
        m = self.mesh
        if prob.gp_kind == "volume":
            if prob.gp_max_order > 0 and (e_minus, axis) in self.volume_gp_patches():
                return self.volume_gp_blocks(e_minus, axis)
            return {(s, t): np.zeros((self.ndof, self.ndof)) for s in range(2) for t in range(2)}
        cells, kap, kavg = self._face_setup(e_minus, axis)
        sgn = (1.0, -1.0)
        xi_face = (1.0, 0.0)
        blocks = {(s, t): np.zeros((self.ndof, self.ndof)) for s in range(2) for t in range(2)}
        gp = m.active_type[cells[0]] == mesh.CUT or m.active_type[cells[1]] == mesh.CUT
        if gp and prob.gp_max_order > 0:
            gx, gw = self.face_quadrature(e_minus, axis, full=True)
            for j in range(1, prob.gp_max_order + 1):
                gam = prob.gp_gamma * prob.h ** (2 * j - 1) / math.factorial(j) ** 2
                N = [self.basis_at(cells[s], gx, axis, j, fixed=(axis, xi_face[s]))
                     for s in range(2)]
                for s in range(2):
                    for t in range(2):
                        blocks[(s, t)] += gam * kavg * sgn[s] * sgn[t] * (N[s].T @ (gw[:, None] * N[t]))
        return blocks

    def face_blocks(self, e_minus, axis):
        """SIPG (DG only) + ghost-penalty blocks of one interior face."""
        b = self.gp_blocks(e_minus, axis)
        if self.discretization == "cg":
            return b
        a = self.sipg_blocks(e_minus, axis)
        return {key: a[key] + b[key] for key in a}

    # ----------------------------------------------------------------- global operator
    def faces_of(self, e):
        """(axis, side, neighbour) of every face of e shared with an active cell."""
        out = []
        for axis in range(self.prob.dim):
            for side in range(2):
                nb = self.mesh.neighbor(e, axis, side)
                if nb >= 0:
                    out.append((axis, side, nb))
        return out

    def assemble(self):
        """Global sparse matrix (small meshes only)."""
        nd = self.ndof
        rows, cols, vals = [], [], []

        def add(ea, eb, blk):
            r = np.repeat(np.arange(nd) + ea * nd, nd)
            c = np.tile(np.arange(nd) + eb * nd, nd)
            rows.append(r)
            cols.append(c)
            vals.append(blk.reshape(-1))

        for e in range(self.mesh.n_active):
            add(e, e, self.cell_matrix(e))
            for axis in range(self.prob.dim):
                ep = self.mesh.neighbor(e, axis, 1)
                if ep < 0:
                    continue
                blocks = self.face_blocks(e, axis)
                cells = (e, ep)
                for (s, t), blk in blocks.items():
                    add(cells[s], cells[t], blk)
        n = self.mesh.n_dofs
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n, n)).tocsr()
        A.sum_duplicates()
        return A

    def apply_rows(self, x, cells, transpose=False):
        """Rows of y = A x (or y = A^T x) that belong to the listed active cells, computed one
        cell at a time.  Returns an array of shape (len(cells), n^d)."""
        nd = self.ndof
        X = np.asarray(x, dtype=np.float64).reshape(-1, nd)
        out = np.zeros((len(cells), nd))
        for r, e in enumerate(cells):
            Ae = self.cell_matrix(e)
            y = (Ae.T if transpose else Ae) @ X[e]
            for axis, side, nb in self.faces_of(e):
                e_minus = e if side == 1 else nb
                s = 0 if side == 1 else 1
                blocks = self.face_blocks(e_minus, axis)
                if transpose:
                    y += blocks[(s, s)].T @ X[e] + blocks[(1 - s, s)].T @ X[nb]
                else:
                    y += blocks[(s, s)] @ X[e] + blocks[(s, 1 - s)] @ X[nb]
            out[r] = y
        return out

    def kappa_gradient(self, x, r, cells=None):
        """dk_K = r^T A_K x with A_K = dA/dkappa_K (A is linear in kappa: A = sum_K kappa_K A_K),
        by the definition: kappa set to the indicator of K, rows of K and of its neighbours."""
        if cells is None:
            cells = range(self.mesh.n_active)
        nd = self.ndof
        R = np.asarray(r, dtype=np.float64).reshape(-1, nd)
        saved = self.mesh.kappa.copy()
        out = []
        try:
            for K in cells:
                self.mesh.kappa[:] = 0.0
                self.mesh.kappa[K] = 1.0
                rows = [K] + [nb for _, _, nb in self.faces_of(K)]
                Y = self.apply_rows(x, rows)
                out.append(float(sum(R[c] @ Y[i] for i, c in enumerate(rows))))
        finally:
            self.mesh.kappa[:] = saved
        return np.array(out)

    # ----------------------------------------------------------------- continuous Q_p
    def cg_numbering(self):
        """Global node of every (active cell, local DoF): lattice point p I_a + i_a, nodes of the
        active cells numbered lexicographically (x fastest).  Returns (n_cg, loc2glob[n_active, nd])."""
        p = self.prob.degree
        d = self.prob.dim
        dims = [p * N + 1 for N in self.prob.n_cells]
        lat = np.zeros((self.mesh.n_active, self.ndof), dtype=np.int64)
        stride = 1
        for a in range(d):
            lat += (self.mesh.active_idx[:, a:a + 1] * p + self.lidx[None, :, a]) * stride
            stride *= dims[a]
        used, loc2glob = np.unique(lat, return_inverse=True)
        return len(used), loc2glob.reshape(lat.shape)

    def cg_prolongation(self):
        n_cg, l2g = self.cg_numbering()
        n_loc = l2g.size
        return sp.csr_matrix((np.ones(n_loc), (np.arange(n_loc), l2g.reshape(-1))), shape=(n_loc, n_cg))

    def cg_matrix(self):
        """A_cg = P^T A_loc P with A_loc the cell-local operator (no SIPG) and P the map from
        global nodes to cell-local DoFs."""
        P = self.cg_prolongation()
        return (P.T @ self.assemble() @ P).tocsr()

    def load_vector(self, f=1.0):
        """b_l = int_{K cap Omega} f phi_l for every cell-local DoF; f is a constant or a function
        of the points (array [m, d] -> [m])."""
        out = np.zeros((self.mesh.n_active, self.ndof))
        for e in range(self.mesh.n_active):
            vx, vw, _, _, _ = self.cell_quadrature(e)
            if len(vw):
                fv = f(vx) if callable(f) else f
                out[e] = (vw * fv) @ self.basis_at(e, vx)
        return out.reshape(-1)

    def l2_error(self, x, u):
        """(||u_h - u||_{L2(Omega)}, ||u||_{L2(Omega)}) for the discrete function with DoF values
        x (cell-local for "dg", global for "cg") and the function u of the points, on the cell
        quadrature of every active cell."""
        xl = self.cg_prolongation() @ x if self.discretization == "cg" else np.asarray(x)
        xl = xl.reshape(self.mesh.n_active, self.ndof)
        err2 = 0.0
        nrm2 = 0.0
        for e in range(self.mesh.n_active):
            vx, vw, _, _, _ = self.cell_quadrature(e)
            if not len(vw):
                continue
            uh = self.basis_at(e, vx) @ xl[e]
            ue = u(vx)
            err2 += vw @ ((uh - ue) ** 2)
            nrm2 += vw @ (ue ** 2)
        return math.sqrt(err2), math.sqrt(nrm2)

    def cg_load_vector(self, f=1.0):
        return self.cg_prolongation().T @ self.load_vector(f)
