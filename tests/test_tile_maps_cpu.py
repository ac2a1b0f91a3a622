"""Index maps of the 3D transfer kernels, replayed on the host for every block
of a launch (no GPU): the tile restriction (32 x 8 x 2 fine cells per block,
one coarse cell per summing thread) writes every coarse cell exactly once from
exactly its children, and the two-plane prolongation updates every fine cell
once, reading only coarse values its block staged. The shapes include odd
sides, whose last coarse cell has one child on that axis (ragged levels)."""
import itertools

import pytest

GX, GY = 32, 8


def nb(n, b):
    return (n + b - 1) // b


SHAPES = [(16, 16, 16), (20, 24, 40), (9, 11, 13), (33, 17, 5), (64, 8, 2), (7, 5, 3)]


@pytest.mark.parametrize("fine", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_tile_restriction_covers_every_coarse_cell_once(fine):
    nx, ny, nz = fine
    cnx, cny, cnz = nb(nx, 2), nb(ny, 2), nb(nz, 2)
    nby = nb(ny, GY)
    written = {}
    for bx, byz in itertools.product(range(nb(nx, GX)), range(nby * cnz)):
        K, by = divmod(byz, nby)
        # phase 1: the fine cells whose residuals this block computes
        tile = set()
        for ty, tx, q in itertools.product(range(GY), range(GX), range(2)):
            i, j, k = bx * GX + tx, by * GY + ty, 2 * K + q
            if i < nx and j < ny and k < nz:
                tile.add((i, j, k))
        # phase 2: threads 0..63 sum children
        for t in range((GX // 2) * (GY // 2)):
            ti, tj = t % (GX // 2), t // (GX // 2)
            I, J = bx * (GX // 2) + ti, by * (GY // 2) + tj
            if I >= cnx or J >= cny:
                continue
            kids = [(2 * I + a, 2 * J + b, 2 * K + c) for c in range(2) for b in range(2) for a in range(2)
                    if 2 * I + a < nx and 2 * J + b < ny and 2 * K + c < nz]
            assert set(kids) <= tile                      # read from this block's shared tile
            assert (2 * tj + 1) < GY and (2 * ti + 1) < GX
            assert (I, J, K) not in written
            written[(I, J, K)] = kids
    assert len(written) == cnx * cny * cnz
    # every fine cell is the child of exactly one coarse cell
    allk = [c for kids in written.values() for c in kids]
    assert len(allk) == len(set(allk)) == nx * ny * nz


@pytest.mark.parametrize("fine", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_two_plane_prolongation_reads_only_staged_values(fine):
    nx, ny, nz = fine
    cnx, cny, cnz = nb(nx, 2), nb(ny, 2), nb(nz, 2)
    SX, SY = GX // 2 + 2, GY // 2 + 2
    nby = nb(ny, GY)
    updated = set()
    for bx, byz in itertools.product(range(nb(nx, GX)), range(nby * cnz)):
        K, by = divmod(byz, nby)
        x0, y0 = bx * GX, by * GY
        X0, Y0 = x0 // 2 - 1, y0 // 2 - 1
        staged = set()
        for t in range(3 * SY * SX):          # the staging loop (stride 256)
            q, rem = divmod(t, SY * SX)
            yy, xx = divmod(rem, SX)
            X, Y, Z = X0 + xx, Y0 + yy, K - 1 + q
            if 0 <= X < cnx and 0 <= Y < cny and 0 <= Z < cnz:
                staged.add((X, Y, Z))
        for ty, tx, q in itertools.product(range(GY), range(GX), range(2)):
            i, j, k = x0 + tx, y0 + ty, 2 * K + q
            if not (i < nx and j < ny and k < nz):
                continue
            assert (i, j, k) not in updated
            updated.add((i, j, k))
            # the coarse cells the interpolation may read: parent and, per axis,
            # the neighbour on the child's side when it exists
            reads = []
            for a, (p, n_c) in enumerate(((i, cnx), (j, cny), (k, cnz))):
                par = p // 2
                nbr = par + 1 if p & 1 else par - 1
                reads.append([par] + ([nbr] if 0 <= nbr < n_c else []))
            for X, Y, Z in itertools.product(*reads):
                assert (X, Y, Z) in staged
                assert 0 <= X - X0 < SX and 0 <= Y - Y0 < SY and 0 <= Z - K + 1 < 3
    assert len(updated) == nx * ny * nz
