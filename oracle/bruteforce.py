"""Dense brute-force restatement of the scheme for tiny grids — TEST INFRASTRUCTURE.

A second oracle, independent of ``fdtd_oracle.c``: the Laplacian is assembled as
an explicit matrix from 1D second-difference matrices (Kronecker sums), the time
stepping is the matrix recurrence of App. E.2 (Eq. cerjan_pde, centred), and the
velocity Jacobian of the gather comes from FORWARD-mode differentiation of that
recurrence (one tangent direction per cell), so J^T r checks the C oracle's
reverse-mode gradient without sharing its derivation.

Inputs are the padded per-cell c = v^2 dt^2 and eta (damping) arrays, on-grid
source/receiver cells, and the wavelet. Grids must be tiny (a few hundred cells).
"""
import numpy as np

D2W = np.array([-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0])


def second_difference(n, h, mirror_low=False):
    """1D 8th-order second-difference matrix on n cells: p = 0 beyond the ends,
    or an odd mirror p(-k) = -p(k) below index 0 when ``mirror_low``."""
    D = np.zeros((n, n))
    for i in range(n):
        for m in range(-4, 5):
            j = i + m
            w = D2W[abs(m)] / (h * h)
            if 0 <= j < n:
                D[i, j] += w
            elif j < 0 and mirror_low:
                D[i, -j] -= w
    return D


def laplacian_matrix(dims, h, free_surface=False):
    """Dense L on the padded grid, dims = (NZ, NX) or (NZ, NY, NX), row-major."""
    if len(dims) == 2:
        nz, nx = dims
        Dz = second_difference(nz, h, free_surface)
        Dx = second_difference(nx, h)
        return np.kron(Dz, np.eye(nx)) + np.kron(np.eye(nz), Dx)
    nz, ny, nx = dims
    Dz = second_difference(nz, h, free_surface)
    Dy = second_difference(ny, h)
    Dx = second_difference(nx, h)
    return (np.kron(np.kron(Dz, np.eye(ny)), np.eye(nx)) +
            np.kron(np.kron(np.eye(nz), Dy), np.eye(nx)) +
            np.kron(np.eye(nz * ny), Dx))


def simulate(L, c, eta, v, dt, wavelet, src_cell, src_scale, rec_cells, surface_rows,
             tangent=False):
    """Run the recurrence (1+a) p+ = 2p - (1-a) p- + c (L p + s), a = eta v^2 dt/2,
    with s = wavelet[n] * src_scale at src_cell. Cells in ``surface_rows`` are
    held at zero. Returns the gather (nt, nrec) and, with ``tangent``, the
    Jacobian dg/dv_k for every padded cell k as an array (nt, nrec, ncell)."""
    n = c.size
    c = c.ravel()
    eta = eta.ravel()
    v = v.ravel()
    a = eta * v * v * dt / 2.0
    da = eta * v * dt           # d a_k / d v_k
    dc = 2.0 * v * dt * dt      # d c_k / d v_k
    nt = len(wavelet)
    pm = np.zeros(n)
    p = np.zeros(n)
    keep = np.ones(n)
    keep[surface_rows] = 0.0
    if tangent:
        Tm = np.zeros((n, n))
        T = np.zeros((n, n))
    g = np.zeros((nt, len(rec_cells)))
    J = np.zeros((nt, len(rec_cells), n)) if tangent else None
    for it in range(nt):
        g[it] = p[rec_cells]
        if tangent:
            J[it] = T[rec_cells]
        s = np.zeros(n)
        s[src_cell] = wavelet[it] * src_scale
        Lp = L @ p
        pn = (2.0 * p - (1.0 - a) * pm + c * (Lp + s)) / (1.0 + a)
        pn *= keep
        if tangent:
            # d/dv_k of the update; the direction-k column only perturbs cell k
            rhs = 2.0 * T - (1.0 - a)[:, None] * Tm + c[:, None] * (L @ T)
            rhs += np.diag(da * (pm - pn) + dc * (Lp + s))
            Tn = rhs / (1.0 + a)[:, None]
            Tn *= keep[:, None]
            Tm, T = T, Tn
        pm, p = p, pn
    return g, J


def replication_matrix(interior, nb, ndim):
    """F with F[padded_cell, interior_cell] = 1 where the padded cell copies
    that interior cell (nearest interior cell in each axis)."""
    if ndim == 2:
        nz, nx = interior
        NZ, NX = nb[0] + nz + nb[1], nb[4] + nx + nb[5]
        F = np.zeros((NZ * NX, nz * nx))
        for z in range(NZ):
            for x in range(NX):
                iz = min(max(z - nb[0], 0), nz - 1)
                ix = min(max(x - nb[4], 0), nx - 1)
                F[z * NX + x, iz * nx + ix] = 1.0
        return F
    nz, ny, nx = interior
    NZ, NY, NX = nb[0] + nz + nb[1], nb[2] + ny + nb[3], nb[4] + nx + nb[5]
    F = np.zeros((NZ * NY * NX, nz * ny * nx))
    for z in range(NZ):
        for y in range(NY):
            for x in range(NX):
                iz = min(max(z - nb[0], 0), nz - 1)
                iy = min(max(y - nb[2], 0), ny - 1)
                ix = min(max(x - nb[4], 0), nx - 1)
                F[(z * NY + y) * NX + x, (iz * ny + iy) * nx + ix] = 1.0
    return F
