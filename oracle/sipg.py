"""SIPG discretisation of -div(kappa grad u) = f on [0,1]^d, homogeneous Dirichlet.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Bilinear form (paper Eq. weak_form_IP, Sec. 2.3.1), read as the symmetric
interior penalty method (theta = -1 in the paper's sign convention) and extended
to a cellwise-constant coefficient kappa_K:

  a(u,v) = sum_K kappa_K (grad u, grad v)_K
         + sum_{F interior} kappa_F [ -<{d_n u},[v]> - <{d_n v},[u]> + gamma_F <[u],[v]> ]
         + sum_{F boundary} kappa_K [ -<d_n u, v>   - <d_n v, u>   + gamma_F <u, v> ]

with n = n_F pointing from K^- to K^+ (+axis for interior facets, outward on the
boundary, Sec. 2.1), [w] = w^- - w^+, {w} = (w^- + w^+)/2, kappa_F the harmonic
mean 2 k^- k^+ / (k^- + k^+) and gamma_F = 2 p (p+1) / h_perp on every facet.
Scaling all facet terms of an interior facet by the harmonic mean is the
weighted-average (SWIP) form of the kappa extension; for kappa = 1 it is the
paper's form exactly.

Layout: u[cell, node], cell = ix + nx*(iy + ny*iz), node = i + q*(j + q*k)
(x fastest), GLL nodes per axis. ``Mesh.grid`` views a vector with shape
(nz, ny, nx, q, q, q) (2D: (ny, nx, q, q)).
"""
import itertools
import numpy as np
import scipy.sparse as sp

from . import refelem

THETA = -1.0  # symmetric interior penalty in the paper's sign convention


class Mesh:
    """Uniform tensor-product mesh of the unit box with n[dir] cells along axis dir
    (the axis-aligned Cartesian cells of Sec. 2.1, uniformly refined) and the
    degree-p tensor-product DG space on it (Sec. 2.2.1)."""

    def __init__(self, n, p, penalty_p=None, basis="gll"):
        """penalty_p: degree whose penalty 2 p (p+1) / h the facets use (default p).
        A lower level of a gradual p-hierarchy keeps the finest level's penalty:
        its operator is then the Galerkin restriction of the finest operator.
        basis: nodes of the Lagrange basis, "gll" (default) or "gl" (Sec. 6.4)."""
        self.n = tuple(int(v) for v in n)
        self.d = len(self.n)
        if self.d not in (2, 3):
            raise ValueError("d must be 2 or 3")
        self.p = int(p)
        self.penalty_p = self.p if penalty_p is None else int(penalty_p)
        self.q = self.p + 1
        self.h = tuple(1.0 / v for v in self.n)
        self.ncell = int(np.prod(self.n))
        self.nloc = self.q ** self.d
        self.ndof = self.ncell * self.nloc
        self.basis = basis
        self.nodes = refelem.basis_nodes(self.p, basis)
        Mr = refelem.mass_1d(self.p, basis)
        Kr = refelem.stiffness_1d(self.p, basis)
        self.M = [Mr * (h / 2.0) for h in self.h]          # 1D mass on a cell of width h
        self.K = [Kr * (2.0 / h) for h in self.h]          # 1D stiffness
        self.e0, self.ep = refelem.endpoint_values(self.p, basis)
        d0, dp = refelem.endpoint_derivs(self.p, basis)
        self.d0 = [d0 * (2.0 / h) for h in self.h]         # physical d/dx at the low end
        self.dp = [dp * (2.0 / h) for h in self.h]         # physical d/dx at the high end

    def gamma(self, direction):
        """Penalty gamma_F = 2 p (p+1) / h for a facet normal to ``direction`` (Sec. 2.3.1)
        (p = penalty_p)."""
        return 2.0 * self.penalty_p * (self.penalty_p + 1) / self.h[direction]

    # axis bookkeeping of the grid view
    def cell_axis(self, direction):
        """Array axis of the cells along ``direction`` (storage layout, no passage)."""
        return self.d - 1 - direction

    def node_axis(self, direction):
        """Array axis of the cell-local nodes along ``direction`` (storage layout)."""
        return 2 * self.d - 1 - direction

    def grid(self, u):
        """DoF vector as the array [cells (z, y, x)][nodes (z, y, x)] (storage layout)."""
        return np.asarray(u, dtype=np.float64).reshape(self.n[::-1] + (self.q,) * self.d)

    def flat(self, U):
        """Inverse of ``grid``: [cell][local node] (storage layout)."""
        return U.reshape(self.ncell, self.nloc)

    def kappa_grid(self, kappa):
        """Per-cell kappa as an array over the cells (kappa = 1 when None)."""
        if kappa is None:
            return np.ones(self.n[::-1])
        return np.asarray(kappa, dtype=np.float64).reshape(self.n[::-1])

    def node_coords(self):
        """Physical coordinates of every DoF, shape (ndof, d): the nodes of Sec. 2.2.1
        mapped to each cell."""
        xi01 = (self.nodes + 1.0) / 2.0
        out = np.zeros((self.ncell, self.nloc, self.d))
        cells = np.indices(self.n[::-1]).reshape(self.d, -1)[::-1]   # (ix, iy, iz) per cell
        nodes = np.indices((self.q,) * self.d).reshape(self.d, -1)[::-1]
        for a in range(self.d):
            out[:, :, a] = (cells[a][:, None] + xi01[nodes[a]][None, :]) * self.h[a]
        return out.reshape(-1, self.d)


def _sl(nd, ax, s):
    idx = [slice(None)] * nd
    idx[ax] = s
    return tuple(idx)


def apply_1d(A, U, ax):
    """Apply the 1D matrix A (rows: output index, cols: input index) along axis ax
    (one factor of a tensor-product operator, Sec. 4.1 "Structure of block-matrices")."""
    return np.moveaxis(np.tensordot(A, U, axes=([1], [ax])), 0, ax)


def _contract(U, vec, ax):
    """sum_i vec[i] U[..., i, ...] along axis ax, keeping ax with length 1."""
    shape = [1] * U.ndim
    shape[ax] = len(vec)
    return np.sum(U * np.asarray(vec).reshape(shape), axis=ax, keepdims=True)


def _lift(F, vec, ax, nd):
    """Outer product inserting ``vec`` along axis ax of a face field with length-1 axis ax."""
    shape = [1] * nd
    shape[ax] = len(vec)
    return F * np.asarray(vec).reshape(shape)


def _tangential_mass(mesh, F, direction):
    """Apply the facet mass matrix (tensor product of 1D masses over the tangential axes)."""
    for t in range(mesh.d):
        if t != direction:
            F = apply_1d(mesh.M[t], F, mesh.node_axis(t))
    return F


# ---------------------------------------------------------------------------
# Assembled route: the bilinear form integrated by quadrature, entry by entry.
# Paper Sec. 2.3.2 (block-sparse matrix A, Eq. matrix_form_IP). Tiny meshes only.
# ---------------------------------------------------------------------------

def _basis_tables(mesh):
    xg, wg = refelem.gauss_legendre(mesh.q)
    V = refelem.lagrange_values(mesh.nodes, xg)           # (q, ng)
    D = refelem.lagrange_derivs(mesh.nodes, xg)
    Ve = refelem.lagrange_values(mesh.nodes, np.array([-1.0, 1.0]))   # (q, 2)
    De = refelem.lagrange_derivs(mesh.nodes, np.array([-1.0, 1.0]))
    return xg, wg, V, D, Ve, De


def local_volume_matrix(mesh):
    """(grad phi_b, grad phi_a)_K for kappa = 1 by d-dimensional Gauss quadrature: the
    volume term of Eq. weak_form_IP (Sec. 2.3.1)."""
    d, q = mesh.d, mesh.q
    xg, wg, V, D, _, _ = _basis_tables(mesh)
    ng = len(xg)
    loc = list(itertools.product(range(q), repeat=d))     # a = (a_x, a_y, a_z)
    pts = list(itertools.product(range(ng), repeat=d))
    nl = len(loc)
    phi = np.zeros((nl, len(pts)))
    grad = np.zeros((d, nl, len(pts)))
    W = np.zeros(len(pts))
    for g, gi in enumerate(pts):
        W[g] = np.prod([wg[gi[a]] * mesh.h[a] / 2.0 for a in range(d)])
        for ia, a in enumerate(loc):
            phi[ia, g] = np.prod([V[a[t], gi[t]] for t in range(d)])
            for k in range(d):
                grad[k, ia, g] = np.prod([(D[a[t], gi[t]] * 2.0 / mesh.h[t]) if t == k else V[a[t], gi[t]]
                                          for t in range(d)])
    Kl = np.einsum('g,kag,kbg->ba', W, grad, grad)
    # reorder from itertools order (a_x slowest) to node = a_x + q a_y + q^2 a_z
    perm = np.array([sum(a[t] * q ** t for t in range(d)) for a in loc])
    out = np.zeros((nl, nl))
    out[np.ix_(perm, perm)] = Kl
    return out


def local_facet_tables(mesh, direction):
    """Values and normal (+axis) derivatives of all cell basis functions on a facet
    normal to ``direction``, at the facet's tangential Gauss points (the facet
    integrals of Eq. weak_form_IP_facets, Sec. 4.1).

    Returns (W, val_lo, der_lo, val_hi, der_hi): the facet quadrature weights and,
    for the cell face at xi_dir = -1 (lo) and +1 (hi), arrays (nloc, npts)."""
    d, q = mesh.d, mesh.q
    xg, wg, V, D, Ve, De = _basis_tables(mesh)
    ng = len(xg)
    tang = [t for t in range(d) if t != direction]
    pts = list(itertools.product(range(ng), repeat=d - 1))
    W = np.array([np.prod([wg[g[i]] * mesh.h[tang[i]] / 2.0 for i in range(d - 1)]) for g in pts])
    res = []
    for end in (0, 1):
        val = np.zeros((mesh.nloc, len(pts)))
        der = np.zeros((mesh.nloc, len(pts)))
        for node in range(mesh.nloc):
            a = [(node // q ** t) % q for t in range(d)]
            for ig, g in enumerate(pts):
                tv = np.prod([V[a[tang[i]], g[i]] for i in range(d - 1)])
                val[node, ig] = Ve[a[direction], end] * tv
                der[node, ig] = De[a[direction], end] * (2.0 / mesh.h[direction]) * tv
        res.append((val, der))
    return W, res[0][0], res[0][1], res[1][0], res[1][1]


def assemble(mesh, kappa=None):
    """Assemble A (scipy CSR, ndof x ndof) from the bilinear form Eq. weak_form_IP by
    quadrature (its matrix, Sec. 2.3.2).

    Rows are test functions, columns trial functions. Cells and facets are
    visited one by one; each facet contributes its four (interior) or one
    (boundary) coupling blocks, exactly as the weak form is written."""
    kap = mesh.kappa_grid(kappa).reshape(-1)
    nl = mesh.nloc
    Kvol = local_volume_matrix(mesh)
    rows, cols, vals = [], [], []

    def add(cr, cc, blk):
        """Scatter one coupling block into the COO lists."""
        r = cr * nl + np.arange(nl)
        c = cc * nl + np.arange(nl)
        rr, cc2 = np.meshgrid(r, c, indexing='ij')
        rows.append(rr.ravel())
        cols.append(cc2.ravel())
        vals.append(blk.ravel())

    for c in range(mesh.ncell):
        add(c, c, kap[c] * Kvol)

    cell_ids = np.arange(mesh.ncell).reshape(mesh.n[::-1])
    for direction in range(mesh.d):
        W, vlo, dlo, vhi, dhi = local_facet_tables(mesh, direction)
        g = mesh.gamma(direction)
        # interior facet: K^- contributes its hi face, K^+ its lo face; n_F = +axis
        side = {'m': (vhi, dhi, +1.0), 'p': (vlo, dlo, -1.0)}   # (value, d/dn, jump sign)
        blocks = {}
        for sb in 'mp':
            for sa in 'mp':
                vb, db, jb = side[sb]
                va, da, ja = side[sa]
                # a(phi_a, phi_b) facet part: -{dn phi_a}[phi_b] - {dn phi_b}[phi_a] + g [phi_a][phi_b]
                blk = (-0.5 * np.einsum('g,ag,bg->ba', W, da, jb * vb)
                       - 0.5 * np.einsum('g,bg,ag->ba', W, db, ja * va)
                       + g * np.einsum('g,ag,bg->ba', W, ja * va, jb * vb))
                blocks[(sb, sa)] = blk
        # boundary facets: outward normal -axis at x=0 (lo face), +axis at x=1 (hi face)
        bnd = {}
        for key, (v, dd, s) in {'lo': (vlo, dlo, -1.0), 'hi': (vhi, dhi, +1.0)}.items():
            dn = s * dd
            bnd[key] = (-np.einsum('g,ag,bg->ba', W, dn, v)
                        - np.einsum('g,bg,ag->ba', W, dn, v)
                        + g * np.einsum('g,ag,bg->ba', W, v, v))
        ca = mesh.cell_axis(direction)
        nd = mesh.n[direction]
        for f in range(nd + 1):
            if 0 < f < nd:
                cm = cell_ids[_sl(mesh.d, ca, f - 1)].ravel()
                cp = cell_ids[_sl(mesh.d, ca, f)].ravel()
                for a_, b_ in zip(cm, cp):
                    kf = 2.0 * kap[a_] * kap[b_] / (kap[a_] + kap[b_])
                    add(a_, a_, kf * blocks[('m', 'm')])
                    add(a_, b_, kf * blocks[('m', 'p')])
                    add(b_, a_, kf * blocks[('p', 'm')])
                    add(b_, b_, kf * blocks[('p', 'p')])
            elif f == 0:
                for c in cell_ids[_sl(mesh.d, ca, 0)].ravel():
                    add(c, c, kap[c] * bnd['lo'])
            else:
                for c in cell_ids[_sl(mesh.d, ca, nd - 1)].ravel():
                    add(c, c, kap[c] * bnd['hi'])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.ndof, mesh.ndof))
    return A.tocsr()


# ---------------------------------------------------------------------------
# Matrix-free facet route: paper Alg. 2 (three stages) with the auxiliary
# facet variables of Techniques 1 and 2.
# ---------------------------------------------------------------------------

def project(mesh, U):
    """Stage 1: projection variables (Eq. solution_projection, gradient_projection).

    For each direction, facets f = 0..n are stacked along that direction's cell
    axis. Returns per direction (ut_m, ut_p, ud_m, ud_p) = (u~^-, u~^+, u~'^-, u~'^+)
    with u~^- = u^-, u~^+ = -u^+ (the sign convention of the paper) and
    u~'^+- = grad u^+- . n_F. On a boundary facet the interior cell is K^- and n_F
    is the outward normal; the ^+ fields are zero there."""
    out = []
    for direction in range(mesh.d):
        ca, na = mesh.cell_axis(direction), mesh.node_axis(direction)
        nd = mesh.n[direction]
        lo_v = _contract(U, mesh.e0, na)
        hi_v = _contract(U, mesh.ep, na)
        lo_d = _contract(U, mesh.d0[direction], na)
        hi_d = _contract(U, mesh.dp[direction], na)
        shape = list(lo_v.shape)
        shape[ca] = nd + 1
        um, up, dm, dpp = (np.zeros(shape) for _ in range(4))
        nds = mesh.d * 2
        if nd > 1:
            um[_sl(nds, ca, slice(1, nd))] = hi_v[_sl(nds, ca, slice(0, nd - 1))]
            dm[_sl(nds, ca, slice(1, nd))] = hi_d[_sl(nds, ca, slice(0, nd - 1))]
            up[_sl(nds, ca, slice(1, nd))] = -lo_v[_sl(nds, ca, slice(1, nd))]
            dpp[_sl(nds, ca, slice(1, nd))] = lo_d[_sl(nds, ca, slice(1, nd))]
        um[_sl(nds, ca, slice(0, 1))] = lo_v[_sl(nds, ca, slice(0, 1))]
        dm[_sl(nds, ca, slice(0, 1))] = -lo_d[_sl(nds, ca, slice(0, 1))]
        um[_sl(nds, ca, slice(nd, nd + 1))] = hi_v[_sl(nds, ca, slice(nd - 1, nd))]
        dm[_sl(nds, ca, slice(nd, nd + 1))] = hi_d[_sl(nds, ca, slice(nd - 1, nd))]
        out.append((um, up, dm, dpp))
    return out


def facet_kappa(mesh, kappa_grid, direction):
    """kappa_F per facet of ``direction`` (harmonic mean inside, kappa_K on the boundary;
    the coefficient extension of Eq. weak_form_IP read for cellwise kappa, Sec. 2.3.1),
    stacked along the cell axis, broadcastable against the face fields."""
    ca = mesh.cell_axis(direction)
    nd = mesh.n[direction]
    k = kappa_grid
    shape = list(k.shape)
    shape[ca] = nd + 1
    kF = np.zeros(shape)
    if nd > 1:
        km = k[_sl(mesh.d, ca, slice(0, nd - 1))]
        kp = k[_sl(mesh.d, ca, slice(1, nd))]
        kF[_sl(mesh.d, ca, slice(1, nd))] = 2.0 * km * kp / (km + kp)
    kF[_sl(mesh.d, ca, slice(0, 1))] = k[_sl(mesh.d, ca, slice(0, 1))]
    kF[_sl(mesh.d, ca, slice(nd, nd + 1))] = k[_sl(mesh.d, ca, slice(nd - 1, nd))]
    return kF.reshape(kF.shape + (1,) * mesh.d)


def numerical_flux(mesh, proj, own_only=False):
    """Stage 2: flux variables (Eq. numerical_fluxes).

    Interior: w = (u~^- + u~^+)/2 = [u]/2, w' = (u~'^- + u~'^+)/2 = {d_n u}.
    Boundary: w = u~^-, w' = u~'^-.
    Returns per direction the fields seen from the K^- side and from the K^+
    side; they are the same unless ``own_only``, in which case each side sees
    the flux of its own projection only (the other side's set to zero). That
    is how the diagonal block A_KK (Schur complement block) is isolated."""
    out = []
    for direction in range(mesh.d):
        um, up, dm, dpp = proj[direction]
        ca = mesh.cell_axis(direction)
        nd = mesh.n[direction]
        nds = 2 * mesh.d
        z = np.zeros_like(um)
        if own_only:
            wm, wdm = 0.5 * (um + z), 0.5 * (dm + z)
            wp, wdp = 0.5 * (z + up), 0.5 * (z + dpp)
        else:
            wm, wdm = 0.5 * (um + up), 0.5 * (dm + dpp)
            wp, wdp = wm, wdm
        for f in (0, nd):                      # boundary facets
            s = _sl(nds, ca, slice(f, f + 1))
            wm = wm.copy(); wdm = wdm.copy(); wp = wp.copy(); wdp = wdp.copy()
            wm[s] = um[s]
            wdm[s] = dm[s]
            wp[s] = um[s]
            wdp[s] = dm[s]
        out.append((wm, wdm, wp, wdp))
    return out


def volume_term(mesh, U, kappa_grid):
    """kappa_K (grad u, grad v)_K for all cells (the cell term of Eq. cell_equation,
    Alg. 2 stage 3): sum over directions of the 1D
    stiffness along that direction and 1D masses along the others."""
    Y = np.zeros_like(U)
    for direction in range(mesh.d):
        T = U
        for a in range(mesh.d):
            T = apply_1d(mesh.K[a] if a == direction else mesh.M[a], T, mesh.node_axis(a))
        Y += T
    return Y * kappa_grid.reshape(kappa_grid.shape + (1,) * mesh.d)


def cell_equation(mesh, U, kappa_grid, flux):
    """Stage 3 left-hand side: A_cc u + A_cf w per cell, Eq. weak_form_IP_facet_spaces:

      (A u)_K = kappa_K (grad u, grad v)_K
              + sum_{F in F(K)} sigma kappa_F ( <v w'> - theta <w grad v . n_K> - gbar <w v> ),

    sigma = -n_K . n_F, gbar = 2 gamma inside, gamma on the boundary."""
    Y = volume_term(mesh, U, kappa_grid)
    nds = 2 * mesh.d
    for direction in range(mesh.d):
        ca, na = mesh.cell_axis(direction), mesh.node_axis(direction)
        nd = mesh.n[direction]
        g = mesh.gamma(direction)
        wm, wdm, wp, wdp = flux[direction]
        kF = facet_kappa(mesh, kappa_grid, direction)
        gbar = np.full(nd + 1, 2.0 * g)
        gbar[0] = gbar[nd] = g
        gshape = [1] * nds
        gshape[ca] = nd + 1
        gbar = gbar.reshape(gshape)
        # hi face of each cell: facet f = i+1, the cell is K^-; n_K = n_F = +axis, sigma = -1
        s_hi = _sl(nds, ca, slice(1, nd + 1))
        W, Wd = _tangential_mass(mesh, wm[s_hi], direction), _tangential_mass(mesh, wdm[s_hi], direction)
        sigma, nK = -1.0, +1.0
        Y += sigma * kF[s_hi] * (_lift(Wd, mesh.ep, na, nds)
                                 - THETA * nK * _lift(W, mesh.dp[direction], na, nds)
                                 - gbar[s_hi] * _lift(W, mesh.ep, na, nds))
        # lo face of each cell: facet f = i; interior: the cell is K^+, n_F = +axis,
        # n_K = -axis, sigma = +1; boundary f = 0: the cell is K^-, n_F = n_K, sigma = -1
        s_lo = _sl(nds, ca, slice(0, nd))
        w_lo, wd_lo = wp[s_lo].copy(), wdp[s_lo].copy()
        s0 = _sl(nds, ca, slice(0, 1))
        w_lo[s0], wd_lo[s0] = wm[s0], wdm[s0]
        sig = np.ones(nd)
        sig[0] = -1.0
        sig = sig.reshape(gbar.shape[:ca] + (nd,) + gbar.shape[ca + 1:])
        W, Wd = _tangential_mass(mesh, w_lo, direction), _tangential_mass(mesh, wd_lo, direction)
        nK = -1.0
        Y += sig * kF[s_lo] * (_lift(Wd, mesh.e0, na, nds)
                               - THETA * nK * _lift(W, mesh.d0[direction], na, nds)
                               - gbar[s_lo] * _lift(W, mesh.e0, na, nds))
    return Y


def apply(mesh, u, kappa=None, own_only=False):
    """A u by the facet route (Alg. 2 stages 1-3 with b = 0). Flat in, flat out."""
    U = mesh.grid(u)
    kg = mesh.kappa_grid(kappa)
    flux = numerical_flux(mesh, project(mesh, U), own_only=own_only)
    return mesh.flat(cell_equation(mesh, U, kg, flux)).reshape(-1)


def residual(mesh, u, b, kappa=None):
    """r = b - A u (the residual of Eq. block-Jacobi-IP, Sec. 2.3.3)."""
    return np.asarray(b, dtype=np.float64).reshape(-1) - apply(mesh, u, kappa)


def block_diagonal(mesh, kappa=None):
    """Diagonal blocks A_KK, shape (ncell, nloc, nloc), the block diagonal of the
    Schur complement S = A_cc + A_cf A_ff A_fc (Sec. 4.1): column j of every
    block is the cell equation applied to the j-th unit vector in every cell,
    with each cell seeing only its own facet projections."""
    B = np.zeros((mesh.ncell, mesh.nloc, mesh.nloc))
    for j in range(mesh.nloc):
        u = np.zeros((mesh.ncell, mesh.nloc))
        u[:, j] = 1.0
        B[:, :, j] = apply(mesh, u, kappa, own_only=True).reshape(mesh.ncell, mesh.nloc)
    return B


class BlockJacobi:
    """Block-Jacobi smoother u <- u + omega A_KK^{-1} (b - A u) (Eq. block-Jacobi-IP),
    with A_KK the exact diagonal blocks (or, with ``interior_only``, Technique 4:
    the block of an interior cell with the cell's own kappa used everywhere)."""

    def __init__(self, mesh, kappa=None, interior_only=False):
        self.mesh = mesh
        self.kappa = None if kappa is None else np.asarray(kappa, dtype=np.float64).reshape(-1)
        if interior_only:
            big = Mesh(tuple(3 for _ in range(mesh.d)), mesh.p, penalty_p=mesh.penalty_p, basis=mesh.basis)
            big.h = mesh.h
            big.M, big.K, big.d0, big.dp = mesh.M, mesh.K, mesh.d0, mesh.dp
            Bi = block_diagonal(big)[(3 ** mesh.d) // 2]
            kap = np.ones(mesh.ncell) if self.kappa is None else self.kappa
            self.B = kap[:, None, None] * Bi[None]
        else:
            self.B = block_diagonal(mesh, self.kappa)
        self.Binv = np.linalg.inv(self.B)

    def apply_inverse(self, r):
        """A_KK^-1 r cell by cell (the block inverse of Eq. block-Jacobi-IP)."""
        R = np.asarray(r).reshape(self.mesh.ncell, self.mesh.nloc)
        return np.einsum('cij,cj->ci', self.Binv, R).reshape(-1)

    def step_alg2(self, u, b, omega, nsteps=1):
        """nsteps of Alg. 2: each step recomputes the projections from u."""
        u = np.array(u, dtype=np.float64).reshape(-1)
        for _ in range(nsteps):
            u = u + omega * self.apply_inverse(residual(self.mesh, u, b, self.kappa))
        return u

    def step_alg4(self, u, b, omega, nsteps=1):
        """nsteps of Alg. 4: one warm-up projection, then per step and cell the
        residual from the stored projections, the update, and the re-projection
        of the updated cell (Technique 5, shift-and-fuse). Returns (u, projections)."""
        mesh = self.mesh
        kg = mesh.kappa_grid(self.kappa)
        U = mesh.grid(np.array(u, dtype=np.float64))
        Bg = mesh.grid(np.asarray(b, dtype=np.float64))
        proj = project(mesh, U)                                    # warm-up traversal
        for _ in range(nsteps):
            R = Bg - cell_equation(mesh, U, kg, numerical_flux(mesh, proj))
            U = U + omega * mesh.grid(self.apply_inverse(mesh.flat(R)))
            proj = project(mesh, U)                                # fused re-projection
        return mesh.flat(U).reshape(-1), proj


# ---------------------------------------------------------------------------
# Right-hand side and error measures (Sec. 6 and 6.1)
# ---------------------------------------------------------------------------

def load_vector(mesh, f, nquad=None):
    """b_i = (f, phi_i) (right-hand side of Eq. weak_form_IP, Sec. 2.3.1) with (p+2)^d
    Gauss-Legendre points per cell. ``f`` takes
    d coordinate arrays and returns values."""
    m = mesh.q + 1 if nquad is None else nquad
    xg, wg = refelem.gauss_legendre(m)
    V = refelem.lagrange_values(mesh.nodes, xg)                 # (q, m)
    d = mesh.d
    coords = []
    for a in range(d):
        idx = np.arange(mesh.n[a])
        pts = (idx[:, None] + (xg[None, :] + 1.0) / 2.0) * mesh.h[a]     # (n_a, m)
        coords.append(pts)
    # grid of quadrature points, shape n[::-1] + (m,)*d
    shp = mesh.n[::-1] + (m,) * d
    X = []
    for a in range(d):
        s = [1] * (2 * d)
        s[mesh.cell_axis(a)] = mesh.n[a]
        s[mesh.node_axis(a)] = m
        X.append(np.broadcast_to(coords[a].reshape(s), shp))
    F = f(*X)
    for a in range(d):
        wshape = [1] * (2 * d)
        wshape[mesh.node_axis(a)] = m
        F = F * (wg * mesh.h[a] / 2.0).reshape(wshape)
    for a in range(d):
        F = apply_1d(V, F, mesh.node_axis(a))
    return mesh.flat(F).reshape(-1)


def l2_error(mesh, u, uex, nquad=None):
    """|| u_h - u_exact ||_{L2(Omega)} with (p+3)^d Gauss points per cell (the error
    measure of Sec. 6.1)."""
    m = mesh.q + 2 if nquad is None else nquad
    xg, wg = refelem.gauss_legendre(m)
    V = refelem.lagrange_values(mesh.nodes, xg)                 # (q, m)
    d = mesh.d
    U = mesh.grid(u)
    for a in range(d):
        U = apply_1d(V.T, U, mesh.node_axis(a))
    shp = mesh.n[::-1] + (m,) * d
    X = []
    for a in range(d):
        idx = np.arange(mesh.n[a])
        pts = (idx[:, None] + (xg[None, :] + 1.0) / 2.0) * mesh.h[a]
        s = [1] * (2 * d)
        s[mesh.cell_axis(a)] = mesh.n[a]
        s[mesh.node_axis(a)] = m
        X.append(np.broadcast_to(pts.reshape(s), shp))
    E = (U - uex(*X)) ** 2
    for a in range(d):
        wshape = [1] * (2 * d)
        wshape[mesh.node_axis(a)] = m
        E = E * (wg * mesh.h[a] / 2.0).reshape(wshape)
    return float(np.sqrt(E.sum()))
