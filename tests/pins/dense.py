"""The walk operator as an explicit dense matrix (brute force on tiny lattices).

Column (c, v) of U is the image of the basis state |v, c>: the coin spreads it
over |v, r> with weights C_v[r, c], then the shift sends each |v, r> to
|v + e_r, r> (moving) or |v + e_r, r xor 1> (flip-flop); a closed link keeps the
amplitude on v in the coin slot the link leaves empty (r xor 1 for moving, r for
flip-flop); at the lattice edge the link is periodic, closed (segment) or
absorbing (line).  Flat index = c * nsites + v (coin-major planes).
"""
import numpy as np

DIR_1D = [(-1, 0), (1, 0)]
DIR_2D = [(1, 0), (-1, 0), (0, 1), (0, -1)]
DIR_DIAG = [(1, 1), (1, -1), (-1, 1), (-1, -1)]


def diagonal_shift_matrix(dims):
    """S of the diagonal lattice (periodic): |x, y, c> -> |x + dx_c, y + dy_c, c>."""
    Lx, Ly = dims
    ns = Lx * Ly
    S = np.zeros((4 * ns, 4 * ns))
    for v in range(ns):
        x, y = v % Lx, v // Lx
        for c, (dx, dy) in enumerate(DIR_DIAG):
            u = ((y + dy) % Ly) * Lx + (x + dx) % Lx
            S[c * ns + u, c * ns + v] = 1.0
    return S


def shift_matrix(dims, flipflop=False, bc=0, closed=None, dirs=None):
    """S as a dense 0/1 matrix.  dims = (N,) or (Lx, Ly).  closed: optional
    (ndim, nsites) flags for the link from site (x, y) to (x+1, y) [axis 0] or
    (x, y+1) [axis 1]."""
    ndim = len(dims)
    Lx = dims[0]
    Ly = dims[1] if ndim == 2 else 1
    ns = Lx * Ly
    d = 2 * ndim
    if dirs is None:
        dirs = DIR_1D if ndim == 1 else DIR_2D
    S = np.zeros((d * ns, d * ns))
    for v in range(ns):
        x, y = v % Lx, v // Lx
        for r in range(d):
            dx, dy = dirs[r]
            axis = 0 if dx != 0 else 1
            n = Lx if axis == 0 else Ly
            p = x if axis == 0 else y
            step = dx if axis == 0 else dy
            link_p = p if step > 0 else (p - 1) % n
            lx, ly = (link_p, y) if axis == 0 else (x, link_p)
            is_closed = bool(closed is not None and closed[axis][ly * Lx + lx])
            at_edge = link_p == n - 1
            if at_edge and bc == 1:
                is_closed = True
            if is_closed:
                tgt_v, tgt_r = v, (r if flipflop else r ^ 1)
            elif at_edge and bc == 2:
                continue
            else:
                q = (p + step) % n
                nx, ny = (q, y) if axis == 0 else (x, q)
                tgt_v, tgt_r = ny * Lx + nx, (r ^ 1 if flipflop else r)
            S[tgt_r * ns + tgt_v, r * ns + v] = 1.0
    return S


def coin_matrix(coins, ns, d):
    """Block-diagonal I (x) C_v as a dense matrix, coins: (d, d) or (ns, d, d)."""
    coins = np.asarray(coins, dtype=np.complex128)
    if coins.ndim == 2:
        coins = np.broadcast_to(coins, (ns, d, d))
    Cm = np.zeros((d * ns, d * ns), dtype=np.complex128)
    for v in range(ns):
        for r in range(d):
            for c in range(d):
                Cm[r * ns + v, c * ns + v] = coins[v, r, c]
    return Cm


def walk_matrix(dims, coins, flipflop=False, bc=0, closed=None, dirs=None):
    ndim = len(dims)
    ns = int(np.prod(dims))
    d = 2 * ndim
    return shift_matrix(dims, flipflop, bc, closed, dirs) @ coin_matrix(coins, ns, d)


def apply_power(U, psi, T):
    flat = np.asarray(psi, dtype=np.complex128).reshape(-1)
    return (np.linalg.matrix_power(U, int(T)) @ flat).reshape(np.shape(psi))
