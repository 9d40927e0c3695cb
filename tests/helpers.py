"""Shared helpers for the parity tests (comparison utilities only; no method arithmetic)."""
import numpy as np


def min_image(a, b, L=1.0):
    """a - b mapped to [-L/2, L/2) per component (positions in a periodic box)."""
    L = np.asarray(L, dtype=np.float64).reshape(-1, *([1] * (np.ndim(a) - 1))) if np.ndim(L) else L
    return (a - b + 0.5 * L) % L - 0.5 * L


def face_distance(pos, n, L=(1.0, 1.0, 1.0)):
    """Distance of each particle to the nearest cell face, in cell units (min over axes)."""
    dist = np.full(pos.shape[1], np.inf)
    for q in range(3):
        s = pos[q] * (n[q] / L[q])
        f = s - np.floor(s)
        dist = np.minimum(dist, np.minimum(f, 1.0 - f))
    return dist


def linear_cells(pos, n, L=(1.0, 1.0, 1.0)):
    idx = []
    for q in range(3):
        i = np.floor(pos[q] * (n[q] / L[q])).astype(np.int64)
        idx.append(np.clip(i, 0, n[q] - 1))
    return idx[0] + n[0] * (idx[1] + n[1] * idx[2])


def chunk_keys_from_cells(cells, n, B):
    """Chunk-major Morton keys of linear cell numbers, by plain bit loops."""
    cells = np.asarray(cells, dtype=np.int64)
    i = cells % n[0]
    j = (cells // n[0]) % n[1]
    k = cells // (n[0] * n[1])
    ncx = -(-n[0] // B)
    ncy = -(-n[1] // B)
    chunk = (i // B) + ncx * ((j // B) + ncy * (k // B))
    li, lj, lk = i % B, j % B, k % B
    m = np.zeros_like(cells)
    b = 0
    while (1 << b) < B:
        m |= ((li >> b) & 1) << (3 * b)
        m |= ((lj >> b) & 1) << (3 * b + 1)
        m |= ((lk >> b) & 1) << (3 * b + 2)
        b += 1
    return (chunk * B ** 3 + m).astype(np.uint32)
