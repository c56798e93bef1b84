"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the DDLR method itself: it only builds the
test matrices (finite-difference Laplacians and a finite-volume jump-coefficient
operator, the model problems of Sec. 5.1), the subdomain maps (box partitions
and random per-axis cuts) and the right-hand sides.  Every random number comes
from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), written out below from its
published definition, so that any consumer can regenerate the same inputs.

Matrices are returned as ``(n, rowptr, colind, val)`` with int32 indices,
float64 values, full symmetric storage and strictly ascending columns per row.
Grid points are numbered ``g = x + nx*(y + ny*z)`` (x fastest); Dirichlet
boundary nodes are eliminated, so every grid point is an unknown.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of SplitMix64 seeded with ``seed``.

    Output i (0-based) is mix(seed + (i+1)*gamma) with the published finaliser
    (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31).
    """
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """u = (z >> 11) * 2^-53 in [0, 1) from SplitMix64 output z."""
    z = splitmix64(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def rhs(n: int, seed: int = 0) -> np.ndarray:
    """Right-hand side with entries uniform in [-1, 1), drawn in index order."""
    return 2.0 * uniform01(seed, n) - 1.0


def rhs_block(n: int, nrhs: int, seed: int = 0) -> np.ndarray:
    """``nrhs`` right-hand sides (column r uses seed+r), shape (n, nrhs)."""
    return np.stack([rhs(n, seed + r) for r in range(nrhs)], axis=1)


def _coo_to_csr(n, rows, cols, vals):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return (n, rowptr.astype(np.int32), cols.astype(np.int32),
            vals.astype(np.float64))


def laplacian(shape) -> tuple:
    """Unscaled 3/5/7-point Laplacian on a 1-D/2-D/3-D grid, Dirichlet boundary.

    Diagonal 2*dim, off-diagonals -1 (the centred-difference model problem of
    Sec. 5.1 with h^2 scaled out).
    """
    shape = tuple(int(s) for s in shape)
    dims = len(shape)
    nx = shape[0]
    ny = shape[1] if dims > 1 else 1
    nz = shape[2] if dims > 2 else 1
    n = nx * ny * nz
    g = np.arange(n, dtype=np.int64)
    x = g % nx
    y = (g // nx) % ny
    z = g // (nx * ny)
    rows = [g]
    cols = [g]
    vals = [np.full(n, 2.0 * dims)]
    steps = [(x, nx, 1)]
    if dims > 1:
        steps.append((y, ny, nx))
    if dims > 2:
        steps.append((z, nz, nx * ny))
    for coord, ext, stride in steps:
        lo = coord > 0
        hi = coord < ext - 1
        rows += [g[lo], g[hi]]
        cols += [g[lo] - stride, g[hi] + stride]
        vals += [np.full(lo.sum(), -1.0), np.full(hi.sum(), -1.0)]
    return _coo_to_csr(n, np.concatenate(rows), np.concatenate(cols),
                       np.concatenate(vals))


def shifted_laplacian(shape, sigma: float) -> tuple:
    """The Laplacian of ``laplacian(shape)`` minus sigma I: the symmetric
    indefinite model problem -Lap u - c u of Sec. 5.1 (c > 0) with h^2 scaled
    out, indefinite once sigma exceeds the smallest eigenvalue."""
    n, rp, ci, va = laplacian(shape)
    va = va.copy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    va[rows == ci] -= float(sigma)
    return n, rp, ci, va


def nine_point(N: int, sigma: float = 0.0) -> tuple:
    """2-D N x N 9-point stencil: diagonal 8 - sigma, -1 to the 8 neighbours
    (Dirichlet).  Its graph has triangles, unlike the 5/7-point Laplacians,
    so incomplete factorisations on its pattern have update terms inside the
    pattern."""
    rows, cols, vals = [], [], []
    for y in range(N):
        for x in range(N):
            i = y * N + x
            rows.append(i); cols.append(i); vals.append(8.0 - sigma)
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if (dx or dy) and 0 <= x + dx < N and 0 <= y + dy < N:
                        rows.append(i); cols.append((y + dy) * N + x + dx); vals.append(-1.0)
    return _coo_to_csr(N * N, np.array(rows), np.array(cols), np.array(vals))


def box_partition(shape, parts) -> tuple[np.ndarray, int]:
    """Split each grid axis into ``parts[a]`` equal ranges (cut at floor(i*N/P)).

    Returns ``(part, p)`` with part[g] = box index, boxes numbered x fastest.
    """
    cuts = [np.floor(np.arange(P + 1) * N / P).astype(np.int64)
            for N, P in zip(shape, parts)]
    return _part_from_cuts(shape, cuts)


def _part_from_cuts(shape, cuts):
    shape = tuple(int(s) for s in shape)
    dims = len(shape)
    n = int(np.prod(shape))
    g = np.arange(n, dtype=np.int64)
    coords = []
    stride = 1
    for a in range(dims):
        coords.append((g // stride) % shape[a])
        stride *= shape[a]
    part = np.zeros(n, dtype=np.int64)
    mult = 1
    for a in range(dims):
        idx = np.searchsorted(cuts[a], coords[a], side="right") - 1
        part += idx * mult
        mult *= len(cuts[a]) - 1
    return part.astype(np.int32), int(mult)


def random_cut_partition(N: int = 96, parts_per_axis: int = 5, seed: int = 0,
                         wmin: int = 8, wmax: int = 32) -> tuple[np.ndarray, int]:
    """Irregular box partition of an N^3 grid: per axis, ``parts_per_axis-1`` cut
    positions drawn uniformly from 1..N-1 (SplitMix64 stream ``seed``, one
    axis after the other), redrawn as a set until every width lies in
    [wmin, wmax].
    """
    ncut = parts_per_axis - 1
    cuts = []
    counter = 0
    for _axis in range(3):
        while True:
            z = splitmix64(seed, ncut, start=counter)
            counter += ncut
            pos = np.sort((z % np.uint64(N - 1)).astype(np.int64) + 1)
            c = np.concatenate([[0], pos, [N]])
            w = np.diff(c)
            if np.all(w >= wmin) and np.all(w <= wmax):
                cuts.append(c)
                break
    return _part_from_cuts((N, N, N), cuts)


def jump_coefficient_fv(N: int = 96, block: int = 8, seed: int = 0,
                        umin: float = -3.0, umax: float = 3.0) -> tuple:
    """7-point finite-volume diffusion on an N^3 cell grid (h = 1).

    Cell coefficient kappa = 10^u, u uniform in [umin, umax) per block^3 group
    of cells (blocks numbered x fastest, drawn in that order).  The
    transmissibility between neighbouring cells is the harmonic mean
    2*k_i*k_j/(k_i+k_j); a Dirichlet boundary face contributes 2*k_i to the
    diagonal.
    """
    nb = N // block
    u = umin + (umax - umin) * uniform01(seed, nb ** 3)
    kb = 10.0 ** u
    n = N ** 3
    g = np.arange(n, dtype=np.int64)
    x = g % N
    y = (g // N) % N
    z = g // (N * N)
    kap = kb[(x // block) + nb * ((y // block) + nb * (z // block))]
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for coord, stride in ((x, 1), (y, N), (z, N * N)):
        for side in (-1, 1):
            inside = (coord > 0) if side < 0 else (coord < N - 1)
            gi = g[inside]
            gj = gi + side * stride
            t = 2.0 * kap[gi] * kap[gj] / (kap[gi] + kap[gj])
            rows.append(gi)
            cols.append(gj)
            vals.append(-t)
            diag[gi] += t
            bnd = ~inside
            diag[g[bnd]] += 2.0 * kap[g[bnd]]
    rows.append(g)
    cols.append(g)
    vals.append(diag)
    return _coo_to_csr(n, np.concatenate(rows), np.concatenate(cols),
                       np.concatenate(vals))


def to_dense(A) -> np.ndarray:
    n, rp, ci, va = A
    D = np.zeros((n, n))
    for i in range(n):
        D[i, ci[rp[i]:rp[i + 1]]] = va[rp[i]:rp[i + 1]]
    return D


def to_scipy(A):
    import scipy.sparse as sps
    n, rp, ci, va = A
    return sps.csr_matrix((va, ci, rp), shape=(n, n))


# Named workloads with the shapes of the paper's model problems (Sec. 5.1).
def workload(name: str):
    """Return ``dict(A=..., part=..., p=..., shape=...)`` for a named workload.

    lap2d_64_b2x2  : 2-D 64x64 5-point Laplacian, 2x2 boxes (n=4,096)
    lap3d_64_b4    : 3-D 64^3 7-point Laplacian, 4^3 boxes (n=262,144)
    lap3d_128_b8   : 3-D 128^3 7-point Laplacian, 8^3 boxes (n=2,097,152)
    jump3d_96_cut5 : 3-D 96^3 jump-coefficient FV, 5x5x5 random cuts
    lap3d_E        : 3-D E^3 Laplacian with (E/16)^3 boxes, E in {32,48,64,96,128}
    indef3d_64_s3e-2 : 3-D 64^3 Laplacian minus 3e-2 I, 4x4x2 boxes (32)
    indef2d_128_s1e-1: 2-D 128^2 Laplacian minus 1e-1 I, 2x1 boxes (2)
    """
    if name == "lap2d_64_b2x2":
        shape = (64, 64)
        A = laplacian(shape)
        part, p = box_partition(shape, (2, 2))
    elif name == "lap3d_64_b4":
        shape = (64, 64, 64)
        A = laplacian(shape)
        part, p = box_partition(shape, (4, 4, 4))
    elif name == "lap3d_128_b8":
        shape = (128, 128, 128)
        A = laplacian(shape)
        part, p = box_partition(shape, (8, 8, 8))
    elif name == "jump3d_96_cut5":
        shape = (96, 96, 96)
        A = jump_coefficient_fv(96, 8, 0)
        part, p = random_cut_partition(96, 5, 0)
    elif name == "indef3d_64_s3e-2":
        shape = (64, 64, 64)
        A = shifted_laplacian(shape, 3e-2)
        part, p = box_partition(shape, (4, 4, 2))
    elif name == "indef2d_128_s1e-1":
        shape = (128, 128)
        A = shifted_laplacian(shape, 1e-1)
        part, p = box_partition(shape, (2, 1))
    elif name.startswith("lap3d_") and name[6:].isdigit():
        e = int(name[6:])
        shape = (e, e, e)
        A = laplacian(shape)
        part, p = box_partition(shape, (e // 16,) * 3)
    else:
        raise KeyError(name)
    return dict(A=A, part=part, p=p, shape=shape)
