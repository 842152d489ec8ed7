"""hp-multigrid around the SIPG block-Jacobi smoother (paper Sec. 5).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* p-transfer (Sec. 5.1, Eq. prolongation): the coarse space is continuous Q1 on
  the same mesh, with unknowns at the interior vertices (homogeneous Dirichlet
  imposed strongly). P maps vertex values to the DG nodal values of the same
  function; the restriction is R = P^T.
* CG levels (Sec. 2.4, Sec. 5.2): A_0 = P^T A P (equal to the kappa-weighted Q1
  stiffness, a pinned fact), A_{l+1} = P_h^T A_l P_h with P_h the nested Q1
  interpolation; point Jacobi with D = diag(A_l).
* h-coarsening: every axis with more than f cells is coarsened by the factor f
  (2 by default; the paper's spacetree uses 3). Coarse vertices sit at fine
  vertex indices 0, f, 2f, ... plus the last vertex n, so a mesh whose cell
  count is not divisible by f gets one shorter coarse cell at the end; the
  spaces stay nested. Coarsening stops once no axis has more than f cells.
* Coarsest level: dense Cholesky solve (FP64).
* V(nu_pre, nu_post) cycle used as preconditioner of FP64 CG, and the paper's
  MGMult (Alg. 7: nu pre-smoothing steps, no post-smoothing, one h-V-cycle for
  the coarse correction, preconditioned-residual exit). The MGMult iteration is
  pinned against its dense cycle matrix; its cycle counts against Tables 3-5
  rest on a reading of omega, nu and gamma, which the paper does not state.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import refelem, sipg


def interior_vertex_count(n):
    """Unknowns of the Q1 space with strong Dirichlet conditions: the interior
    vertices (Sec. 2.2.3, 2.4)."""
    return int(np.prod([v - 1 for v in n]))


def p_prolongation(mesh):
    """P (ndof x nvert): value at every DG node of the Q1 hat of each interior
    vertex of the cell (products of 1D hats (1-xi)/2, (1+xi)/2): the
    p-prolongation of Eq. prolongation (Sec. 5.1)."""
    d, q = mesh.d, mesh.q
    m = [v - 1 for v in mesh.n]
    xi = mesh.nodes
    hat = [(1.0 - xi) / 2.0, (1.0 + xi) / 2.0]
    cells = np.indices(mesh.n[::-1]).reshape(d, -1)[::-1]          # (ix, iy, iz)
    cid = np.arange(mesh.ncell)
    rows, cols, vals = [], [], []
    for node in range(mesh.nloc):
        a = [(node // q ** t) % q for t in range(d)]
        for corner in range(2 ** d):
            c = [(corner >> t) & 1 for t in range(d)]
            v = [cells[t] + c[t] for t in range(d)]                 # vertex index per axis
            ok = np.ones(mesh.ncell, dtype=bool)
            for t in range(d):
                ok &= (v[t] >= 1) & (v[t] <= mesh.n[t] - 1)
            vid = np.zeros(mesh.ncell, dtype=np.int64)
            stride = 1
            for t in range(d):
                vid += (v[t] - 1) * stride
                stride *= m[t]
            w = np.prod([hat[c[t]][a[t]] for t in range(d)])
            rows.append(cid[ok] * mesh.nloc + node)
            cols.append(vid[ok])
            vals.append(np.full(ok.sum(), w))
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.ndof, interior_vertex_count(mesh.n)))
    return P.tocsr()


def q1_stiffness(n, kappa=None):
    """kappa-weighted Q1 stiffness on the interior vertices, assembled cell by cell
    from the element integrals (grad hat_a, grad hat_b) by 2-point Gauss quadrature
    (Eq. weak_form_cg, Sec. 2.4)."""
    d = len(n)
    h = [1.0 / v for v in n]
    xg, wg = np.polynomial.legendre.leggauss(2)
    hat = lambda c, x: (1.0 - x) / 2.0 if c == 0 else (1.0 + x) / 2.0
    dhat = lambda c, x: -0.5 if c == 0 else 0.5
    Ke = np.zeros((2 ** d, 2 ** d))
    import itertools
    for gi in itertools.product(range(2), repeat=d):
        W = np.prod([wg[gi[t]] * h[t] / 2.0 for t in range(d)])
        for A_ in range(2 ** d):
            ca = [(A_ >> t) & 1 for t in range(d)]
            for B_ in range(2 ** d):
                cb = [(B_ >> t) & 1 for t in range(d)]
                s = 0.0
                for k in range(d):
                    ga = np.prod([dhat(ca[t], xg[gi[t]]) * 2.0 / h[t] if t == k else hat(ca[t], xg[gi[t]])
                                  for t in range(d)])
                    gb = np.prod([dhat(cb[t], xg[gi[t]]) * 2.0 / h[t] if t == k else hat(cb[t], xg[gi[t]])
                                  for t in range(d)])
                    s += ga * gb
                Ke[B_, A_] += W * s
    ncell = int(np.prod(n))
    kap = np.ones(ncell) if kappa is None else np.asarray(kappa, dtype=np.float64).reshape(-1)
    m = [v - 1 for v in n]
    cells = np.indices(tuple(n)[::-1]).reshape(d, -1)[::-1]
    vids, oks = [], []
    for corner in range(2 ** d):
        c = [(corner >> t) & 1 for t in range(d)]
        v = [cells[t] + c[t] for t in range(d)]
        ok = np.ones(ncell, dtype=bool)
        vid = np.zeros(ncell, dtype=np.int64)
        stride = 1
        for t in range(d):
            ok &= (v[t] >= 1) & (v[t] <= n[t] - 1)
            vid += (v[t] - 1) * stride
            stride *= m[t]
        vids.append(vid)
        oks.append(ok)
    rows, cols, vals = [], [], []
    for A_ in range(2 ** d):
        for B_ in range(2 ** d):
            ok = oks[A_] & oks[B_]
            rows.append(vids[B_][ok])
            cols.append(vids[A_][ok])
            vals.append(kap[ok] * Ke[B_, A_])
    nv = interior_vertex_count(n)
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nv, nv)).tocsr()


def coarse_positions(n, f):
    """Fine vertex indices that are coarse vertices along one axis: 0, f, 2f, ..., n
    (the h-coarsening of Sec. 5.2, factor f)."""
    pos = list(range(0, n, f))
    pos.append(n)
    return pos


def can_coarsen(v, f):
    """An axis with v cells is coarsened only if at least two coarse cells remain
    (the stop rule of the h-coarsening, Sec. 5.2)."""
    return v > f


def coarsen_n(n, f):
    """Cells per axis of the next coarser Q1 mesh (Sec. 5.2)."""
    return tuple(len(coarse_positions(v, f)) - 1 if can_coarsen(v, f) else v for v in n)


def interp_1d(n, f):
    """Nested Q1 interpolation along one axis, interior vertices only:
    (n-1) x (nc-1) with linear weights between neighbouring coarse vertices
    (one factor of the h-prolongation, Sec. 5.2)."""
    if not can_coarsen(n, f):
        return sp.identity(max(n - 1, 0), format='csr')
    pos = coarse_positions(n, f)
    nc = len(pos) - 1
    P = np.zeros((n + 1, nc + 1))
    P[n, nc] = 1.0
    for j in range(nc):
        a, b = pos[j], pos[j + 1]
        for i in range(a, b):                 # fine vertices a <= i < b of coarse cell j
            P[i, j] = (b - i) / (b - a)
            P[i, j + 1] = (i - a) / (b - a)
    return sp.csr_matrix(P[1:n, 1:nc])


def h_prolongation(n, f):
    """P_h between interior-vertex vectors of the meshes n and coarsen_n(n, f)
    (x fastest: the Kronecker product z (x) y (x) x of the 1D interpolations;
    the h-prolongation of Sec. 5.2)."""
    mats = [interp_1d(v, f) for v in n]
    P = mats[0]
    for t in range(1, len(n)):
        P = sp.kron(mats[t], P, format='csr')
    return P


def dg_interp_1d(nodes_f, nodes_c):
    """I[i, j] = l_j^c(x_i^f): the degree-(q_c - 1) Lagrange basis on nodes_c at
    the fine nodes (exact injection of the coarse polynomial space; the nested DG
    spaces of the gradual p-coarsening the outlook of Sec. 6.3 proposes)."""
    return refelem.lagrange_values(nodes_c, nodes_f).T


def dg_p_prolongation(mesh_f, mesh_c):
    """P (ndof_f x ndof_c): cellwise injection of the degree p_c DG space into
    the degree p_f space on the same mesh, the tensor product of interp_1d along
    every axis (node index x fastest; Sec. 6.3 outlook)."""
    I1 = dg_interp_1d(mesh_f.nodes, mesh_c.nodes)
    Pc = I1
    for _ in range(mesh_f.d - 1):
        Pc = np.kron(I1, Pc)                          # (z, y, x) ordering: x fastest
    return sp.kron(sp.identity(mesh_f.ncell, format="csr"), sp.csr_matrix(Pc), format="csr")


class Hierarchy:
    """The DG level(s) plus the CG levels of the hp hierarchy.

    gradual=False: the paper's hierarchy, DG degree p straight to continuous Q1.
    gradual=True: DG degrees p, p-1, ..., 1, then continuous Q1 (the nested
    sequence V_DG^p > V_DG^(p-1) > ... > V_CG^1 of the paper's outlook,
    Sec. 6.3). Every lower DG level keeps the finest penalty, so its operator is
    the Galerkin product P^T A P of the level above; it is smoothed with its own
    block Jacobi (nu_pre, nu_post steps)."""

    def __init__(self, mesh, kappa=None, factor=2, nu_pre=2, nu_post=2,
                 omega_dg=None, omega_cg=None, interior_only=False, gradual=False):
        self.mesh = mesh
        self.kappa = None if kappa is None else np.asarray(kappa, dtype=np.float64).reshape(-1)
        self.nu_pre, self.nu_post = nu_pre, nu_post
        self.omega_dg = default_omega_dg(mesh.d) if omega_dg is None else omega_dg
        self.omega_cg = default_omega_cg(mesh.d) if omega_cg is None else omega_cg
        self.smoother = sipg.BlockJacobi(mesh, self.kappa, interior_only=interior_only)
        # lower DG levels (gradual p-coarsening)
        self.dg_meshes, self.dg_smoothers, self.Pdg = [mesh], [self.smoother], []
        if gradual:
            for pc in range(mesh.p - 1, 0, -1):
                mc = sipg.Mesh(mesh.n, pc, penalty_p=mesh.penalty_p, basis=mesh.basis)
                self.Pdg.append(dg_p_prolongation(self.dg_meshes[-1], mc))
                self.dg_meshes.append(mc)
                self.dg_smoothers.append(sipg.BlockJacobi(mc, self.kappa, interior_only=interior_only))
        self.P = p_prolongation(self.dg_meshes[-1])
        self.ns = [mesh.n]
        self.A = [q1_stiffness(mesh.n, self.kappa)]
        self.Ph = []
        while any(can_coarsen(v, factor) for v in self.ns[-1]):
            n = self.ns[-1]
            Ph = h_prolongation(n, factor)
            self.Ph.append(Ph)
            self.ns.append(coarsen_n(n, factor))
            self.A.append((Ph.T @ self.A[-1] @ Ph).tocsr())
        self.D = [A.diagonal() for A in self.A]
        Ac = self.A[-1].toarray()
        self.coarse_chol = sla.cho_factor(Ac) if Ac.shape[0] > 0 else None

    @property
    def nlevels(self):
        """Q1 levels below the DG level(s), the coarsest included."""
        return len(self.A)

    def coarse_solve(self, r):
        """Exact solve on the coarsest Q1 level (Alg. 6 coarse solve)."""
        if self.coarse_chol is None:
            return np.zeros(0)
        return sla.cho_solve(self.coarse_chol, r)

    def cg_jacobi(self, level, u, b, nsteps):
        """``nsteps`` damped point-Jacobi steps on a Q1 level (Sec. 2.4 smoother)."""
        A, D = self.A[level], self.D[level]
        for _ in range(nsteps):
            u = u + self.omega_cg * (b - A @ u) / D
        return u

    def vcycle_cg(self, level, b):
        """h-multigrid V-cycle on CG level ``level`` with zero initial guess (Sec. 5.2)."""
        if level == self.nlevels - 1:
            return self.coarse_solve(b)
        u = self.cg_jacobi(level, np.zeros_like(b), b, self.nu_pre)
        r = b - self.A[level] @ u
        e = self.vcycle_cg(level + 1, self.Ph[level].T @ r)
        u = u + self.Ph[level] @ e
        return self.cg_jacobi(level, u, b, self.nu_post)

    def vcycle_dg(self, level, r):
        """V-cycle from DG level ``level`` with zero initial guess: smoothing,
        residual, restriction to the next DG level (or to the CG levels below the
        last DG level), correction, smoothing (Alg. 6 with the smoothing of Alg. 4
        around it, Sec. 5.1)."""
        mesh, sm = self.dg_meshes[level], self.dg_smoothers[level]
        u = np.zeros(mesh.ndof)
        u = sm.step_alg2(u, r, self.omega_dg, self.nu_pre)
        res = sipg.residual(mesh, u, r, self.kappa)
        if level == len(self.dg_meshes) - 1:
            u = u + self.P @ self.vcycle_cg(0, self.P.T @ res)
        else:
            u = u + self.Pdg[level] @ self.vcycle_dg(level + 1, self.Pdg[level].T @ res)
        return sm.step_alg2(u, r, self.omega_dg, self.nu_post)

    def vcycle(self, r):
        """z = V(r): hp V(nu_pre, nu_post) cycle with zero initial guess on the DG level
        (Sec. 5.2)."""
        return self.vcycle_dg(0, r)

    def coarse_grid_correction(self, u, b):
        """Alg. 6: residual, restriction, one (h- or hp-) V-cycle, prolongation."""
        res = sipg.residual(self.mesh, u, b, self.kappa)
        if len(self.dg_meshes) == 1:
            return self.P @ self.vcycle_cg(0, self.P.T @ res)
        return self.Pdg[0] @ self.vcycle_dg(1, self.Pdg[0].T @ res)


def default_omega_dg(d):
    """Default block-Jacobi damping (an input everywhere; the paper gives no value).
    lambda_max(D^-1 A) is just below 2 for the SIPG blocks, so omega < 1 keeps the
    smoother convergent and the symmetric V-cycle positive definite."""
    return 0.8


def default_omega_cg(d):
    """Default point-Jacobi damping on the Q1 levels (lambda_max(D^-1 A) is about
    1.43 in 2D and 1.35 in 3D)."""
    return 0.8


def pcg(hier, b, x0=None, rtol=1e-10, maxit=200, flexible=False):
    """FP64 preconditioned CG with the V-cycle as preconditioner (the multigrid
    cycle as the preconditioner P^-1 of Sec. 5.1 "Exit criterion"; Alg. 7 iterates
    it stationarily, see ``mgmult``). Stops when
    ||b - A x||_2 <= rtol ||b||_2 (recursively updated residual). Returns
    (x, iterations, history of relative residuals)."""
    mesh = hier.mesh
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros(mesh.ndof) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
    r = b - sipg.apply(mesh, x, hier.kappa)
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bn]
    if hist[-1] <= rtol:
        return x, 0, hist
    z = hier.vcycle(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        Ap = sipg.apply(mesh, p, hier.kappa)
        alpha = rz / (p @ Ap)
        x = x + alpha * p
        r_old = r
        r = r - alpha * Ap
        hist.append(np.linalg.norm(r) / bn)
        if hist[-1] <= rtol:
            return x, it, hist
        z = hier.vcycle(r)
        rz_new = r @ z
        beta = ((r - r_old) @ z) / rz if flexible else rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, maxit, hist


def mgmult(hier, b, u0=None, eps=1e-7, maxit=500, residual_kind='unprec'):
    """Alg. 7 (MGMult): nu block-Jacobi steps, coarse-grid correction (Alg. 6,
    one h-V-cycle), until the chosen relative residual drops below eps.
    residual_kind 'unprec': ||b - A u|| / ||b - A u_0||; 'prec':
    ||u - u_old|| / ||u_1 - u_0||. Returns (u, cycles). The iterates are pinned
    against the dense cycle matrix and the exit rules against the norms of those
    iterates (tests); the cycle counts of Tables 3-5 depend on omega, nu and the
    penalty, which the paper does not state (a reading, not a pin)."""
    mesh = hier.mesh
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    u = np.zeros(mesh.ndof) if u0 is None else np.array(u0, dtype=np.float64).reshape(-1)
    r0 = np.linalg.norm(b - sipg.apply(mesh, u, hier.kappa))
    rho1 = None
    for k in range(1, maxit + 1):
        u_old = u
        u = hier.smoother.step_alg2(u, b, hier.omega_dg, hier.nu_pre)
        u = u + hier.coarse_grid_correction(u, b)
        if residual_kind == 'prec':
            rho = np.linalg.norm(u - u_old)
            rho1 = rho if rho1 is None else rho1
            if rho / rho1 < eps:
                return u, k
        else:
            if np.linalg.norm(b - sipg.apply(mesh, u, hier.kappa)) / r0 < eps:
                return u, k
    return u, maxit
