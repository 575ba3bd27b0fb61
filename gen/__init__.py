"""Seeded synthetic inputs for the multifrontal Cholesky path.

This module is shared by the oracle tests, the GPU tests and the benchmark.
It builds matrices, orderings and right-hand sides only; it contains no part
of the factorization or solve arithmetic.

Matrices are returned as full symmetric CSR triples ``(rowptr int64, colind
int32, values float64)`` with sorted column indices.  Orderings are returned as
``perm`` with ``perm[new] = old`` (so ``C = A[perm][:, perm]``).

The workloads stand in for the paper's Albany land-ice meshes and the Xyce
matrices, which are not available (paper Sec. 5, experiment setup):

* ``laplacian_2d``      -- 5-point Dirichlet Laplacian (diag 4, off -1).
* ``laplacian_3d``      -- 7-point Dirichlet Laplacian, optional coefficient
                           jumps per 8^3 block with harmonic-mean edge weights.
* ``q1_extruded``       -- extruded Q1 hexahedral mesh carrying the symmetric
                           first-order-Stokes (Blatter-Pattyn) velocity form with
                           two horizontal components per node plus a basal
                           friction term, the ice-sheet-like stand-in.
* ``nd_perm``           -- geometric nested dissection on a node grid.
* ``box_batch``         -- many independent 3D Laplacian boxes (a batch of
                           subdomains), as a block-diagonal matrix.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "laplacian_1d", "laplacian_2d", "laplacian_3d", "q1_extruded", "nd_perm",
    "random_spd", "random_nonsym", "nonsym_3d", "pivot_nodes_3d", "rhs", "box_batch", "block_diag_csr", "csr_matvec",
    "config1", "config2", "config3", "config5",
]


# --------------------------------------------------------------------------
# CSR helpers (no factorization arithmetic)
# --------------------------------------------------------------------------
def _coo_to_csr(n, rows, cols, vals):
    """Sum duplicates and return sorted full CSR."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    start = np.nonzero(np.concatenate(([True], key[1:] != key[:-1])))[0] if len(key) else key
    uniq = key[start]
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = uniq // n
    c = (uniq % n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(np.bincount(r, minlength=n))
    return rowptr, c, summed.astype(np.float64)


def csr_matvec(rowptr, colind, values, x):
    """y = A x for CSR A (x may be 1D or 2D column-major-ish (n, nrhs))."""
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    x = np.asarray(x)
    if x.ndim == 1:
        return np.bincount(rows, weights=values * x[colind], minlength=n)
    out = np.zeros((n, x.shape[1]))
    for r in range(x.shape[1]):
        out[:, r] = np.bincount(rows, weights=values * x[colind, r], minlength=n)
    return out


def block_diag_csr(mats):
    """Block-diagonal union of CSR matrices (batch of independent subdomains)."""
    rowptrs, cols, vals = [], [], []
    off_n = 0
    off_nnz = 0
    for (rp, ci, v) in mats:
        n = len(rp) - 1
        rowptrs.append(rp[:-1] + off_nnz)
        cols.append(ci.astype(np.int64) + off_n)
        vals.append(v)
        off_n += n
        off_nnz += rp[-1]
    rowptr = np.concatenate(rowptrs + [np.array([off_nnz], dtype=np.int64)])
    return rowptr.astype(np.int64), np.concatenate(cols).astype(np.int32), np.concatenate(vals)


# --------------------------------------------------------------------------
# Structured stencil matrices
# --------------------------------------------------------------------------
def laplacian_1d(n):
    """Tridiagonal [-1, 2, -1] (Dirichlet), natural order."""
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[:-1], i[1:]])
    vals = np.concatenate([np.full(n, 2.0), np.full(n - 1, -1.0), np.full(n - 1, -1.0)])
    return _coo_to_csr(n, rows, cols, vals)


def _grid_laplacian(shape, kappa=None):
    """Nodal-coefficient Dirichlet Laplacian on a grid (x fastest).

    Edge weight between neighbours i, j is the harmonic mean
    2 k_i k_j / (k_i + k_j); each missing (boundary) neighbour adds k_i to the
    diagonal.  With k == 1 this is the standard 2d+1 point Laplacian with
    diagonal 2d and off-diagonal -1.
    """
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    n = int(np.prod(shape))
    if kappa is None:
        kappa = np.ones(n)
    kappa = np.asarray(kappa, dtype=np.float64).reshape(-1)
    # node index = x + Nx*(y + Ny*z)  (x fastest); numpy arrays indexed [z, y, x]
    grid = np.arange(n).reshape(shape[::-1])
    kg = kappa.reshape(shape[::-1])
    diag = np.zeros(shape[::-1])
    rows, cols, vals = [], [], []
    for ax in range(nd):
        npax = nd - 1 - ax  # numpy axis of grid axis `ax`
        sl_a = [slice(None)] * nd
        sl_b = [slice(None)] * nd
        sl_a[npax] = slice(0, shape[ax] - 1)
        sl_b[npax] = slice(1, shape[ax])
        ia = grid[tuple(sl_a)].ravel()
        ib = grid[tuple(sl_b)].ravel()
        ka = kg[tuple(sl_a)]
        kb = kg[tuple(sl_b)]
        w = 2.0 * ka * kb / (ka + kb)
        diag[tuple(sl_a)] += w
        diag[tuple(sl_b)] += w
        w = w.ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-w, -w]
        # boundary (Dirichlet) contributions: first and last layer along ax
        lo = [slice(None)] * nd
        hi = [slice(None)] * nd
        lo[npax] = slice(0, 1)
        hi[npax] = slice(shape[ax] - 1, shape[ax])
        diag[tuple(lo)] += kg[tuple(lo)]
        diag[tuple(hi)] += kg[tuple(hi)]
    idx = grid.ravel()
    rows.append(idx)
    cols.append(idx)
    vals.append(diag.ravel())
    return _coo_to_csr(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def laplacian_2d(nx, ny=None):
    """5-point Dirichlet Laplacian on nx*ny nodes: diagonal 4, off-diagonal -1."""
    ny = nx if ny is None else ny
    return _grid_laplacian((nx, ny))


def laplacian_3d(nx, ny=None, nz=None, jump_block=None, jump_value=1e3, seed=None):
    """7-point Dirichlet Laplacian on nx*ny*nz nodes.

    With ``jump_block=b`` the nodal coefficient is constant on b^3 blocks and is
    1 or ``jump_value`` with probability 1/2 each (seeded), edge weights are
    harmonic means.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    kappa = None
    if jump_block is not None:
        rng = np.random.default_rng(seed)
        bx, by, bz = (-(-nx // jump_block), -(-ny // jump_block), -(-nz // jump_block))
        blocks = np.where(rng.random((bz, by, bx)) < 0.5, 1.0, float(jump_value))
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        kappa = blocks[z // jump_block, y // jump_block, x // jump_block].ravel()
    return _grid_laplacian((nx, ny, nz), kappa)


# --------------------------------------------------------------------------
# Extruded Q1 mesh with the first-order Stokes (Blatter-Pattyn) velocity form
# --------------------------------------------------------------------------
def _q1_reference_matrices(hx, hy, hz):
    """Element matrices of a hx*hy*hz trilinear brick (2x2x2 Gauss).

    Returns (K, M) where K (16x16) is the viscous form for mu = 1 with dof
    ordering (local node, component) and M (8x8) is the bottom-face mass matrix
    (only nodes with c == 0 nonzero).

    Bilinear form for velocity (u, v) and test (phi, psi):
        2 mu [ (2u_x + v_y) phi_x + (u_y + v_x)/2 phi_y + u_z/2 phi_z
             + (u_y + v_x)/2 psi_x + (u_x + 2v_y) psi_y + v_z/2 psi_z ]
    which is symmetric and positive semi-definite.
    """
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    wq = 0.5
    local = [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]

    def l(t, a):
        return t if a else 1.0 - t

    def dl(a):
        return 1.0 if a else -1.0

    K = np.zeros((16, 16))
    vol = hx * hy * hz
    for qx in g:
        for qy in g:
            for qz in g:
                w = wq ** 3 * vol
                grads = []
                for (a, b, c) in local:
                    gx = dl(a) / hx * l(qy, b) * l(qz, c)
                    gy = l(qx, a) * dl(b) / hy * l(qz, c)
                    gz = l(qx, a) * l(qy, b) * dl(c) / hz
                    grads.append((gx, gy, gz))
                for p in range(8):
                    px, py, pz = grads[p]
                    for q in range(8):
                        qx_, qy_, qz_ = grads[q]
                        # (alpha, beta) = (0,0): 4 Nq_x Np_x + Nq_y Np_y + Nq_z Np_z
                        K[2 * p, 2 * q] += w * (4 * qx_ * px + qy_ * py + qz_ * pz)
                        # (1,1): Nq_x Np_x + 4 Nq_y Np_y + Nq_z Np_z
                        K[2 * p + 1, 2 * q + 1] += w * (qx_ * px + 4 * qy_ * py + qz_ * pz)
                        # test comp 0, trial comp 1: 2 Nq_y Np_x + Nq_x Np_y
                        K[2 * p, 2 * q + 1] += w * (2 * qy_ * px + qx_ * py)
                        # test comp 1, trial comp 0: 2 Nq_x Np_y + Nq_y Np_x
                        K[2 * p + 1, 2 * q] += w * (2 * qx_ * py + qy_ * px)
    M = np.zeros((8, 8))
    area = hx * hy
    for qx in g:
        for qy in g:
            w = wq ** 2 * area
            vals = [l(qx, a) * l(qy, b) * (1.0 if c == 0 else 0.0) for (a, b, c) in local]
            for p in range(8):
                for q in range(8):
                    M[p, q] += w * vals[p] * vals[q]
    return K, M


def q1_extruded(ex, ey, ez, hx=1.0, hy=1.0, hz=0.01, beta=1.0, seed=1):
    """Extruded Q1 hexahedral mesh, 2 velocity dofs per node (interleaved).

    ex*ey*ez elements, (ex+1)*(ey+1)*(ez+1) nodes, node index x fastest, dof =
    2*node + component.  Per-element viscosity mu_e = 10**U[-2, 0] (seeded).
    A basal friction term beta * int_{z=0} (u phi + v psi) makes the form SPD.
    Matrix entries between nodes sharing an element are stored even where the
    value cancels (structural pattern = 27-point stencil x 2x2 dof blocks).
    """
    rng = np.random.default_rng(seed)
    mu = 10.0 ** rng.uniform(-2.0, 0.0, size=(ez, ey, ex))
    K, M = _q1_reference_matrices(hx, hy, hz)
    Nx, Ny, Nz = ex + 1, ey + 1, ez + 1
    nn = Nx * Ny * Nz
    n = 2 * nn
    local = [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    lidx = {t: i for i, t in enumerate(local)}
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    # values[z, y, x, d, alpha, beta]
    val = np.zeros((Nz, Ny, Nx, 27, 2, 2))
    # pad mu with zeros outside the element range
    mup = np.zeros((ez + 2, ey + 2, ex + 2))
    mup[1:-1, 1:-1, 1:-1] = mu
    basal = np.zeros((ez + 2, ey + 2, ex + 2))
    basal[1, 1:-1, 1:-1] = beta  # elements in the bottom layer (ez index 0)
    Z, Y, X = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    for di, (dx, dy, dz) in enumerate(offs):
        for (a, b, c) in local:
            qa, qb, qc = a + dx, b + dy, c + dz
            if not (0 <= qa <= 1 and 0 <= qb <= 1 and 0 <= qc <= 1):
                continue
            # element containing node p at local position (a,b,c): e = p - (a,b,c)
            m_e = mup[Z - c + 1, Y - b + 1, X - a + 1]
            f_e = basal[Z - c + 1, Y - b + 1, X - a + 1]
            p = lidx[(a, b, c)]
            q = lidx[(qa, qb, qc)]
            for al in range(2):
                for be in range(2):
                    val[:, :, :, di, al, be] += m_e * K[2 * p + al, 2 * q + be]
                    if al == be:
                        val[:, :, :, di, al, be] += f_e * M[p, q]
    # structural validity of each neighbour
    valid = np.zeros((Nz, Ny, Nx, 27), dtype=bool)
    for di, (dx, dy, dz) in enumerate(offs):
        valid[:, :, :, di] = ((X + dx >= 0) & (X + dx < Nx) & (Y + dy >= 0) & (Y + dy < Ny)
                              & (Z + dz >= 0) & (Z + dz < Nz))
    node = (X + Nx * (Y + Ny * Z)).reshape(-1)
    dnode = np.array([dx + Nx * (dy + Ny * dz) for (dx, dy, dz) in offs], dtype=np.int64)
    valid = valid.reshape(nn, 27)
    val = val.reshape(nn, 27, 2, 2)
    counts = valid.sum(axis=1) * 2  # entries per dof row
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1::2] = counts
    rowptr[2::2] = counts
    rowptr = np.cumsum(rowptr)
    nnz = int(rowptr[-1])
    colind = np.empty(nnz, dtype=np.int32)
    values = np.empty(nnz, dtype=np.float64)
    # columns per node row: for each valid neighbour (sorted by node), beta 0,1
    qnode = node[:, None] + dnode[None, :]  # (nn, 27), increasing along axis 1
    for al in range(2):
        cols_full = np.stack([2 * qnode, 2 * qnode + 1], axis=2)  # (nn, 27, 2)
        vals_full = val[:, :, al, :]
        mask = np.repeat(valid[:, :, None], 2, axis=2)
        cflat = cols_full[mask]
        vflat = vals_full[mask]
        # rows 2*node+al occupy contiguous segments; masks keep row-major order
        starts = rowptr[2 * node + al]
        lens = counts
        dst = np.repeat(starts - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens) + np.arange(lens.sum())
        colind[dst] = cflat.astype(np.int32)
        values[dst] = vflat
    return rowptr, colind, values


def _q1_elasticity_element(h, E, nu):
    """24 x 24 stiffness of a cube Q1 element of side h for isotropic linear
    elasticity (Lame lambda, mu from E, nu), 2 x 2 x 2 Gauss points; local
    node (a, b, c) in {0,1}^3, x fastest, dof = 3 node + component."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(6), np.arange(6)] += np.array([2 * mu, 2 * mu, 2 * mu, mu, mu, mu])
    local = [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    g = [-1 / np.sqrt(3), 1 / np.sqrt(3)]
    K = np.zeros((24, 24))
    for xi in g:
        for eta in g:
            for ze in g:
                B = np.zeros((6, 24))
                for p, (a, b, c) in enumerate(local):
                    sa, sb, sc = 2 * a - 1, 2 * b - 1, 2 * c - 1
                    # derivatives of (1 + s xi)(1 + s eta)(1 + s ze) / 8, times 2 / h
                    dx = sa * (1 + sb * eta) * (1 + sc * ze) / 8 * 2 / h
                    dy = sb * (1 + sa * xi) * (1 + sc * ze) / 8 * 2 / h
                    dz = sc * (1 + sa * xi) * (1 + sb * eta) / 8 * 2 / h
                    B[0, 3 * p] = dx
                    B[1, 3 * p + 1] = dy
                    B[2, 3 * p + 2] = dz
                    B[3, 3 * p], B[3, 3 * p + 1] = dy, dx
                    B[4, 3 * p + 1], B[4, 3 * p + 2] = dz, dy
                    B[5, 3 * p], B[5, 3 * p + 2] = dz, dx
                K += B.T @ D @ B * (h / 2) ** 3
    return K


def elasticity_3d(N, E=1.0, nu=0.3):
    """3D linear elasticity on N^3 nodes of a unit cube of Q1 hexahedra, 3
    dofs per node (interleaved; node index x fastest): the 27-point stencil
    of the paper's FastILU experiments (n = 3 N^3).  The nodes of the face
    x = 0 are clamped: their rows and columns become those of the identity,
    which keeps the matrix SPD."""
    h = 1.0 / (N - 1)
    Ke = _q1_elasticity_element(h, E, nu)
    e = np.arange(N - 1)
    ez, ey, ex = np.meshgrid(e, e, e, indexing="ij")
    base = (ex + N * (ey + N * ez)).reshape(-1)
    local = np.array([a + N * (b + N * c) for c in (0, 1) for b in (0, 1) for a in (0, 1)])
    nodes = base[:, None] + local[None, :]                        # (elements, 8)
    dofs = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(len(base), 24)
    rows = np.repeat(dofs, 24, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, 24)).reshape(-1)
    vals = np.tile(Ke.reshape(-1), len(base))
    n = 3 * N ** 3
    node_of = np.arange(n) // 3
    fixed = (node_of % N) == 0
    keep = ~(fixed[rows] | fixed[cols])
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    fd = np.nonzero(fixed)[0]
    rows = np.concatenate([rows, fd])
    cols = np.concatenate([cols, fd])
    vals = np.concatenate([vals, np.ones(len(fd))])
    return _coo_to_csr(n, rows, cols, vals)


def dense_spd(n, seed=0):
    """Dense SPD matrix as CSR: a_ij = u_ij / (1 + |i - j|) with u_ij =
    u_ji ~ U[0.5, 1] (seeded), a_ii = n (diagonally dominant).  One front of
    n pivot columns: every trailing update is one large dense matrix."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.5, 1.0, size=(n, n))
    u = np.triu(u) + np.triu(u, 1).T
    i = np.arange(n)
    A = u / (1.0 + np.abs(i[:, None] - i[None, :]))
    A[i, i] = float(n)
    rowptr = np.arange(0, n * n + 1, n, dtype=np.int64)
    colind = np.tile(np.arange(n, dtype=np.int32), n)
    return rowptr, colind, A.reshape(-1)


def kkt_3d(nx, ny=None, nz=None, delta=1e-2, seed=0):
    """Symmetric quasi-definite saddle-point matrix on an nx x ny x nz grid,
    2 unknowns per node interleaved (dof 2 i: u_i, 2 i + 1: p_i):
        [ K    B^T     ]
        [ B   -delta I ],
    K the 7-point Dirichlet Laplacian on u, B a node-local coupling of p_i
    to u_i (weight U[1, 2]) and to the grid neighbours of node i (weights
    -U[0.1, 0.3]), seeded.  Indefinite (n/2 negative eigenvalues) but
    quasi-definite, so every symmetric permutation of it has an LDL^T
    factorization with D diagonal."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    kp, kc, kv = laplacian_3d(nx, ny, nz)
    nn = len(kp) - 1
    krow = np.repeat(np.arange(nn, dtype=np.int64), np.diff(kp))
    kcol = kc.astype(np.int64)
    # B has the pattern of K: the diagonal and the neighbours
    bval = np.where(krow == kcol, rng.uniform(1.0, 2.0, len(kv)), -rng.uniform(0.1, 0.3, len(kv)))
    rows = np.concatenate([2 * krow, 2 * krow + 1, 2 * kcol, 2 * np.arange(nn) + 1])
    cols = np.concatenate([2 * kcol, 2 * kcol, 2 * krow + 1, 2 * np.arange(nn) + 1])
    vals = np.concatenate([kv, bval, bval, -delta * np.ones(nn)])
    return _coo_to_csr(2 * nn, rows, cols, vals)


# --------------------------------------------------------------------------
# Geometric nested dissection
# --------------------------------------------------------------------------
def nd_perm(shape, split_axes=None, leaf_nodes=8, dofs=1):
    """Geometric nested dissection ordering of a node grid (x fastest).

    A box is a leaf when it holds <= ``leaf_nodes`` nodes or no splittable axis
    has extent >= 3.  Otherwise it is split along its longest splittable axis
    (ties -> lowest axis index) at mid = lo + size//2; the order is: left part,
    right part, then the separator plane, each plane/leaf in lexicographic
    (x fastest) order.  With ``dofs > 1`` the dofs of a node are consecutive.
    Returns perm with perm[new] = old.
    """
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    if split_axes is None:
        split_axes = tuple(range(nd))
    cache = {}

    def lex(sz):
        """Node indices of a box of size sz in its own numbering (x fastest)."""
        return np.arange(int(np.prod(sz)), dtype=np.int64)

    def local_order(sz):
        # order of the nodes of a box of size sz, as indices of the box's own
        # lexicographic numbering; depends only on the box size
        if sz in cache:
            return cache[sz]
        cand = [a for a in split_axes if sz[a] >= 3]
        if int(np.prod(sz)) <= leaf_nodes or not cand or min(sz) <= 0:
            out = lex(sz)
        else:
            ax = max(cand, key=lambda a: (sz[a], -a))
            mid = sz[ax] // 2
            strides = [1]
            for d in sz[:-1]:
                strides.append(strides[-1] * d)
            parts = []
            for lo, hi in ((0, mid), (mid + 1, sz[ax]), (mid, mid + 1)):
                sub = list(sz)
                sub[ax] = hi - lo
                sub = tuple(sub)
                if min(sub) <= 0:
                    continue
                # coordinates of the sub-box's nodes in its own numbering
                o = local_order(sub) if (lo, hi) != (mid, mid + 1) else lex(sub)
                coords = []
                rem = o
                for d in range(nd):
                    coords.append(rem % sub[d])
                    rem = rem // sub[d]
                coords[ax] = coords[ax] + lo
                idx = np.zeros(len(o), dtype=np.int64)
                for d in range(nd):
                    idx += coords[d] * strides[d]
                parts.append(idx)
            out = np.concatenate(parts) if parts else lex(sz)
        cache[sz] = out
        return out

    perm_nodes = local_order(shape) if int(np.prod(shape)) > 0 else np.zeros(0, dtype=np.int64)
    if dofs == 1:
        return perm_nodes.astype(np.int32)
    p = (perm_nodes[:, None] * dofs + np.arange(dofs)[None, :]).reshape(-1)
    return p.astype(np.int32)


# --------------------------------------------------------------------------
# Random small SPD matrices (symbolic and numeric pins)
# --------------------------------------------------------------------------
def random_spd(n, density=0.1, seed=0, dense_rows=0):
    """Random sparse SPD matrix: random symmetric pattern with a diagonal,
    off-diagonal values U[-1,1], diagonal = row |sum| + U[0.5,1.5]."""
    rng = np.random.default_rng(seed)
    m = rng.random((n, n)) < density
    m = np.triu(m, 1)
    for r in range(min(dense_rows, n)):
        m[r, r + 1:] = True
    iu, ju = np.nonzero(m)
    v = rng.uniform(-1.0, 1.0, size=len(iu))
    rows = np.concatenate([iu, ju])
    cols = np.concatenate([ju, iu])
    vals = np.concatenate([v, v])
    absrow = np.bincount(rows, weights=np.abs(vals), minlength=n)
    d = absrow + rng.uniform(0.5, 1.5, size=n)
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, d])
    return _coo_to_csr(n, rows, cols, vals)


def random_nonsym(n, density=0.1, seed=0, dominance=2.0):
    """Random sparse nonsymmetric matrix with a symmetric pattern: entries
    (i, j) and (j, i) drawn independently from U[-1, 1].  With dominance > 0
    the diagonal is dominance x (the column's off-diagonal |sum|) + U[0.5, 1],
    so C is strictly column diagonally dominant (LU without pivoting exists
    for every symmetric ordering, and partial pivoting swaps nothing); with
    dominance = 0 the diagonal is U[-1, 1] too."""
    rng = np.random.default_rng(seed)
    m = np.triu(rng.random((n, n)) < density, 1)
    iu, ju = np.nonzero(m)
    rows = np.concatenate([iu, ju])
    cols = np.concatenate([ju, iu])
    vals = rng.uniform(-1.0, 1.0, size=len(rows))
    if dominance > 0:
        colsum = np.bincount(cols, weights=np.abs(vals), minlength=n)
        d = dominance * colsum + rng.uniform(0.5, 1.0, size=n)
    else:
        d = rng.uniform(-1.0, 1.0, size=n)
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, d])
    return _coo_to_csr(n, rows, cols, vals)


def nonsym_3d(nx, ny=None, nz=None, wind=2.0, small_diag=0.0, seed=0):
    """7-point convection-diffusion operator -Laplace(u) + w . grad(u) on an
    nx x ny x nz grid (Dirichlet, central differences, unit spacing): entry
    (i, i +- e_a) = -1 +- w_a / 2 with a seeded wind w_a in U[-wind, wind]
    per node and axis, diagonal 6.  The pattern is symmetric, the values are
    not; for |w_a| > 2 the matrix is no longer diagonally dominant.  A
    fraction ``small_diag`` of the diagonal entries (seeded) is replaced by
    U[-0.5, 0.5], so that partial pivoting really swaps rows."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    kp, kc, kv = laplacian_3d(nx, ny, nz)
    n = len(kp) - 1
    row = np.repeat(np.arange(n, dtype=np.int64), np.diff(kp))
    col = kc.astype(np.int64)
    w = rng.uniform(-wind, wind, size=(n, 3))
    off = row != col
    d = col - row
    axis = np.where(np.abs(d) == 1, 0, np.where(np.abs(d) == nx, 1, 2))
    vals = np.where(off, -1.0 + np.sign(d) * w[row, axis] / 2.0, 6.0)
    if small_diag > 0:
        pick = rng.random(n) < small_diag
        dv = np.where(pick, rng.uniform(-0.5, 0.5, size=n), 6.0)
        vals = np.where(off, vals, dv[row])
    return _coo_to_csr(n, row, col, vals)


def pivot_nodes_3d(nx, ny=None, nz=None, dofs=2, seed=0):
    """Node-block matrix that needs pivoting, with a unique pivot sequence:
    A = Pi_0 B on an nx x ny x nz grid with `dofs` unknowns per node
    (dof d i + t), dense dofs x dofs blocks between a node and itself and
    its 7-point neighbours (so every row of a node has the same pattern).
    B is strictly column diagonally dominant (diagonal 4 x the column's
    off-diagonal |sum| + 1, off-diagonal U[-1, 1] x 0.2); Pi_0 reverses the
    dof order inside every node, and the entries of B that Pi_0 puts on
    the diagonal of dof 0 of each node are exactly zero.  So LU without
    pivoting stops at the first column with a zero pivot, while partial
    pivoting within any diagonal block that holds a whole node picks the
    dominant row of B each time: it finds Pi_0 and factors B."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    kp, kc, _ = laplacian_3d(nx, ny, nz)
    nn = len(kp) - 1
    a = np.repeat(np.arange(nn, dtype=np.int64), np.diff(kp))
    b = kc.astype(np.int64)
    t = np.arange(dofs)
    ti, tj = np.meshgrid(t, t, indexing="ij")
    rows = (dofs * a[:, None, None] + ti[None]).ravel()
    cols = (dofs * b[:, None, None] + tj[None]).ravel()
    vals = rng.uniform(-1.0, 1.0, size=rows.shape) * 0.2
    n = dofs * nn
    # the entry of B that lands on the diagonal of (node, dof 0): row
    # (node, dofs - 1), column (node, dof 0)
    same = (rows // dofs == cols // dofs)
    vals[same & (rows % dofs == dofs - 1) & (cols % dofs == 0) & (dofs > 1)] = 0.0
    diag = rows == cols
    vals[diag] = 0.0
    colsum = np.bincount(cols, weights=np.abs(vals), minlength=n)
    vals[diag] = 4.0 * colsum[cols[diag]] + 1.0
    node = rows // dofs
    prow = dofs * node + (dofs - 1 - rows % dofs)  # Pi_0: reverse inside the node
    return _coo_to_csr(n, prow, cols, vals)


def random_perm(n, seed=0):
    return np.random.default_rng(seed).permutation(n).astype(np.int32)


def random_nodes(n, max_size=4, seed=0, scatter=True):
    """Group the n DoFs into nodes of U{1..max_size} DoFs.  Returns node_of
    (node id per DoF, original numbering; with ``scatter`` a node's DoFs are
    spread over the numbering) and a random ordering that keeps each node's
    DoFs consecutive (nodes in random order, DoFs ascending inside)."""
    rng = np.random.default_rng(seed)
    sizes = []
    while sum(sizes) < n:
        sizes.append(int(rng.integers(1, max_size + 1)))
    sizes[-1] -= sum(sizes) - n
    lab = np.repeat(np.arange(len(sizes)), sizes)
    dof = rng.permutation(n) if scatter else np.arange(n)
    node_of = np.empty(n, dtype=np.int32)
    node_of[dof] = lab
    order = rng.permutation(len(sizes))
    perm = np.concatenate([np.sort(np.nonzero(node_of == u)[0]) for u in order]) if n else \
        np.zeros(0, dtype=np.int64)
    return node_of, perm.astype(np.int32)


def rhs(n, nrhs=1, seed=0):
    """Right-hand sides U[-1,1], shape (n,) or (n, nrhs), column-major usable."""
    rng = np.random.default_rng(seed)
    if nrhs == 1:
        return rng.uniform(-1.0, 1.0, size=n)
    return np.asfortranarray(rng.uniform(-1.0, 1.0, size=(n, nrhs)))


def box_batch(count=512, lo=8, hi=48, seed=4, leaf_nodes=8):
    """Batch of 7-point Laplacian boxes with sides U{lo..hi} per axis.

    Returns (list of (rowptr, colind, values, perm), sides).
    """
    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, size=(count, 3))
    out = []
    for (a, b, c) in sides:
        rp, ci, v = laplacian_3d(int(a), int(b), int(c))
        perm = nd_perm((int(a), int(b), int(c)), leaf_nodes=leaf_nodes)
        out.append((rp, ci, v, perm))
    return out, sides


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
def config1():
    """2D 5-point Laplacian 64x64 (n=4096), geometric ND, b ~ U[-1,1] seed 0."""
    rp, ci, v = laplacian_2d(64)
    perm = nd_perm((64, 64))
    return rp, ci, v, perm, rhs(64 * 64, 1, seed=0)


def config2(ex=256, ey=256, ez=10):
    """Extruded Q1 ice-sheet-like mesh, 2 dofs/node, ND on the horizontal plane."""
    rp, ci, v = q1_extruded(ex, ey, ez, seed=1)
    perm = nd_perm((ex + 1, ey + 1, ez + 1), split_axes=(0, 1), dofs=2)
    n = len(rp) - 1
    return rp, ci, v, perm, rhs(n, 1, seed=3)


def config3(N=96, nrhs=1):
    """7-point Laplacian N^3 with 8^3-block coefficient jumps {1, 1e3} (seed 2)."""
    rp, ci, v = laplacian_3d(N, N, N, jump_block=8, jump_value=1e3, seed=2)
    perm = nd_perm((N, N, N))
    return rp, ci, v, perm, rhs(N ** 3, nrhs, seed=3)


def config5(N=64, nrhs=1):
    """Plain 7-point Laplacian N^3 (closed-form log-determinant available)."""
    rp, ci, v = laplacian_3d(N, N, N)
    perm = nd_perm((N, N, N))
    return rp, ci, v, perm, rhs(N ** 3, nrhs, seed=5)
