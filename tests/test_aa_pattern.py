"""The AA in-place streaming pattern of the step kernels, emulated on the host
with the oracle's own single-cell collision, against the oracle's two-array
push streaming -- the addressing the CUDA kernels implement, checked without a
GPU.  And its slab-decomposed form (the multi-GPU design): even steps are local;
an odd step's cells next to a slab face read and write one slot per lattice per
face cell of the neighbouring slab (slot 6 of the layer below, slot 5 of the
layer above), so those slots travel in before and back after each odd step.

AA pattern (D3Q7, one buffer A[lattice, slot, z, y, x]):
  even parity: cell x reads slot (i, x), writes direction i to slot (opp i, x);
  odd parity:  cell x reads slot (opp i, x - c_i), writes direction i to slot (i, x + c_i).
"""
import numpy as np
import pytest

import oracle
from paper_2606_00641_gb300 import fields

C = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]  # (x, y, z)
OPP = [0, 2, 1, 4, 3, 6, 5]
TAU = [0.6, 0.55, 0.55, 0.55, 0.7, 0.6, 0.6, 0.6]


def shift(a, c, sign=1):
    """result[x] = a[x - sign c] over the last three axes (z, y, x), periodic."""
    return np.roll(a, shift=(sign * c[2], sign * c[1], sign * c[0]), axis=(-3, -2, -1))


def collide(F, gamma, cells):
    out = F.copy()
    for z, y, x in cells:
        out[:, :, z, y, x] = oracle.ideal_collide_cell(3, gamma, TAU, F[:, :, z, y, x])
    return out


def all_cells(shape):
    return [(z, y, x) for z in range(shape[0]) for y in range(shape[1]) for x in range(shape[2])]


def aa_step(A, parity, gamma):
    cells = all_cells(A.shape[2:])
    if parity == 0:
        P = collide(A, gamma, cells)
        return P[:, OPP]                      # direction i lands in slot opp i of the same cell
    F = np.stack([shift(A[:, OPP[i]], C[i]) for i in range(7)], axis=1)  # F_i(x) = A[opp i, x - c_i]
    P = collide(F, gamma, cells)
    return np.stack([shift(P[:, i], C[i]) for i in range(7)], axis=1)   # slot (i, x + c_i) = P_i(x)


def logical(A, parity):
    if parity == 0:
        return A
    return np.stack([shift(A[:, OPP[i]], C[i]) for i in range(7)], axis=1)


def setup(shape, seed):
    f0 = fields.ideal_fields(shape, seed, mach=1.0, cfl=0.2)
    return f0, oracle.ideal_init(f0.Q, f0.gamma)


@pytest.mark.parametrize("steps", [1, 2, 5])
def test_aa_in_place_pattern_equals_two_array_streaming(steps):
    shape = (4, 5, 6)
    f0, f = setup(shape, 31)
    A, ref = f.copy(), f.copy()
    for s in range(steps):
        A = aa_step(A, s & 1, f0.gamma)
        ref = oracle.ideal_step(ref, f0.gamma, TAU)
    np.testing.assert_array_equal(logical(A, steps & 1), ref)


def test_slab_decomposed_aa_pattern_equals_the_single_domain():
    # three z-slabs of two layers, each stored with a ghost layer below and above
    shape, slabs = (6, 4, 5), 3
    f0, f = setup(shape, 32)
    zl = shape[0] // slabs
    S = []
    for r in range(slabs):
        ext = np.zeros(f.shape[:2] + (zl + 2,) + shape[1:])
        ext[:, :, 1:zl + 1] = f[:, :, r * zl:(r + 1) * zl]
        S.append(ext)
    interior = [(z, y, x) for z in range(1, zl + 1) for y in range(shape[1]) for x in range(shape[2])]
    moved = 0
    steps = 5
    for s in range(steps):
        if s & 1:
            # odd step: the slots the face layers read and write in the neighbours come in ...
            for r in range(slabs):
                below, above = S[(r - 1) % slabs], S[(r + 1) % slabs]
                S[r][:, 6, 0] = below[:, 6, zl]        # slot 6 of the layer below my bottom layer
                S[r][:, 5, zl + 1] = above[:, 5, 1]    # slot 5 of the layer above my top layer
                moved += 2 * 8 * shape[1] * shape[2]
            new = []
            for r in range(slabs):
                A = S[r]
                F = np.stack([shift(A[:, OPP[i]], C[i]) for i in range(7)], axis=1)
                P = collide(F, f0.gamma, interior)
                B = A.copy()
                for i in range(7):
                    # interior cells write direction i to slot (i, x + c_i), ghost layers included
                    src = shift(P[:, i], C[i])
                    lo, hi = (2, zl + 2) if C[i][2] == 1 else ((0, zl) if C[i][2] == -1 else (1, zl + 1))
                    B[:, i, lo:hi] = src[:, lo:hi]
                new.append(B)
            S = new
            # ... and go back to their owners after the step
            for r in range(slabs):
                below, above = S[(r - 1) % slabs], S[(r + 1) % slabs]
                below[:, 6, zl] = S[r][:, 6, 0]
                above[:, 5, 1] = S[r][:, 5, zl + 1]
                moved += 2 * 8 * shape[1] * shape[2]
        else:
            # even step: every read and write stays in the cell
            for r in range(slabs):
                P = collide(S[r], f0.gamma, interior)
                S[r][:, :, 1:zl + 1] = P[:, OPP, 1:zl + 1]
    got = np.concatenate([S[r][:, :, 1:zl + 1] for r in range(slabs)], axis=2)
    ref = f.copy()
    for _ in range(steps):
        ref = oracle.ideal_step(ref, f0.gamma, TAU)
    np.testing.assert_array_equal(logical(got, steps & 1), ref)
    # two odd steps x (in and out) x (two faces) x slabs: one slot per lattice per face cell each time
    assert moved == 2 * 2 * 2 * slabs * 8 * shape[1] * shape[2]
