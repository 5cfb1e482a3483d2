"""Checks of the seeded input generators against closed forms.

The generators hold no method arithmetic; these tests make sure the inputs
have the geometry the workloads describe (Siddon lengths, bounds ordering,
structure sizes, row-length mix).
"""
import numpy as np
import pytest

import synth


def test_ct_row_sums_equal_chord_lengths():
    """Siddon: a ray's intersection lengths add up to its chord through the
    image square (closed form of the slab clip)."""
    A = synth.ct_matrix(32, 24, 45)
    sums = np.asarray(A.to_scipy().sum(axis=1)).ravel()
    chords = np.array([synth.ct_chord(32, 24, 45, r) for r in range(A.m)])
    np.testing.assert_allclose(sums, chords, atol=1e-5)


def test_ct_axis_aligned_ray_pixel_lengths():
    """At angle 0 a ray through pixel centres crosses N pixels of one image row
    with length equal to the pixel size 2/N."""
    N = 16
    # nbin chosen so that bin offsets hit pixel-row centres: s_k = (k - (nb-1)/2) * 2sqrt2/nb
    A = synth.ct_matrix(N, 1, 45)
    for r in range(A.m):
        s = (r - 22) * (2 * np.sqrt(2) / 45)
        i_row = int(np.floor((s + 1) / (2 / N)))
        cols = A.col[A.row_ptr[r]:A.row_ptr[r + 1]]
        vals = A.val[A.row_ptr[r]:A.row_ptr[r + 1]]
        if abs(s) < 1 and abs((s + 1) / (2 / N) - np.round((s + 1) / (2 / N))) > 1e-6:
            assert len(cols) == N
            np.testing.assert_array_equal(cols, i_row * N + np.arange(N))
            np.testing.assert_allclose(vals, 2 / N, rtol=1e-6)


@pytest.mark.parametrize("maker", ["ct", "seismic"])
def test_columns_sorted_and_in_range(maker):
    if maker == "ct":
        A = synth.ct_matrix(48, 30, 70)
    else:
        seg = synth.seismic_geometry(32, 64, 0.01, 8, 32)
        A = synth.seismic_matrix(32, 64, 0.01, seg)
    assert A.col.min() >= 0 and A.col.max() < A.n
    for i in range(A.m):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    assert np.all(A.val > 0)


def test_seismic_rays_have_segment_lengths():
    """Source-receiver segments lie inside the grid, so row sums equal the
    Euclidean source-receiver distance."""
    seg = synth.seismic_geometry(32, 64, 0.01, 8, 32)
    A = synth.seismic_matrix(32, 64, 0.01, seg)
    sums = np.asarray(A.to_scipy().sum(axis=1)).ravel()
    L = np.hypot(seg[:, 2] - seg[:, 0], seg[:, 3] - seg[:, 1])
    np.testing.assert_allclose(sums, L, rtol=1e-5)


def test_ct_problem_bounds_and_empty_rows():
    P = synth.ct_problem(32, 20, 41)
    assert np.all(P.l <= P.u)
    empty = np.diff(P.A.row_ptr) == 0
    assert empty.any()
    assert np.all(P.l[empty] == 0) and np.all(P.u[empty] == 0)
    assert P.x_true.min() >= 0 and P.x_true.max() <= 1


def test_rt_structure_fractions():
    st = synth.rt_structures(100, 60, 50)
    N = 300000
    assert 0.07 < len(st["target"]) / N < 0.09
    assert 0.09 < len(st["oar1"]) / N < 0.11
    assert 0.09 < len(st["oar2"]) / N < 0.11
    allv = np.concatenate(list(st.values()))
    assert len(np.unique(allv)) == len(allv)


def test_random_problem_row_mix():
    A = synth.random_csr(500, 300, seed=1, mean_len=20, empty_frac=0.1, long_rows=3,
                         long_len=290)
    lens = np.diff(A.row_ptr)
    assert (lens == 0).sum() > 20 and (lens == 290).sum() == 3


def test_line_problem_rows_are_segments_on_the_grid():
    H, W = 96, 211
    p = synth.line_problem(H, W, 400, seed=5)
    A = p.A
    assert p.shape == (H, W) and A.n == H * W and A.m == 400
    assert A.col.min() >= 0 and A.col.max() < H * W
    for i in range(0, A.m, 37):
        j = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(j) > 0)            # sorted, no repeats
        assert 1 <= len(j) <= 80
    q = synth.line_problem(H, W, 400, seed=5)
    assert np.array_equal(q.A.col, A.col) and np.array_equal(q.l, p.l)
    assert np.all(p.l <= p.u)
