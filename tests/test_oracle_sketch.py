"""Pins for the oracle's sparse-sign embedding (Eq. 1; Clarkson-Woodruff sketch of Section 4.1)."""
import os

import numpy as np
import pytest

from oracle import sketch as sk


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_splitmix64_published_outputs():
    # First outputs of SplitMix64 started at state 0, as printed by the published reference implementation (the
    # fixture cites it).
    with open(os.path.join(GOLDEN, "splitmix64_state0.txt")) as f:
        want = [int(line, 16) for line in f if line.strip() and not line.startswith("#")]
    assert len(want) == 3
    got = sk.splitmix64_sequence(0, len(want))
    assert [int(x) for x in got] == want


@pytest.mark.parametrize("seed", [0, 1, 12345, 2**63 + 17])
def test_counter_form_equals_sequential_stream(seed):
    seq = sk.splitmix64_sequence(seed, 64)
    ctr = sk.draw(seed, np.arange(64, dtype=np.uint64))
    assert np.array_equal(seq, ctr)


@pytest.mark.parametrize("n,s,zeta", [(1000, 120, 8), (5000, 400, 8), (777, 16, 8), (300, 9, 8), (64, 8, 8),
                                      (1000, 50, 1)])
def test_pattern_distinct_rows_and_signs(n, s, zeta):
    rows, signs = sk.sparse_sign_pattern(n, s, zeta, seed=1)
    assert rows.shape == (n, zeta) and signs.shape == (n, zeta)
    assert rows.min() >= 0 and rows.max() < s
    srt = np.sort(rows, axis=1)
    assert np.all(np.diff(srt, axis=1) > 0), "rows of a column must be distinct"
    assert set(np.unique(signs).tolist()) <= {-1, 1}


def test_full_column_when_s_equals_zeta():
    # s == zeta forces every column to use every row (exercises the collision retries and the probe fallback)
    rows, _ = sk.sparse_sign_pattern(2000, 8, 8, seed=3)
    assert np.all(np.sort(rows, axis=1) == np.arange(8)[None, :])


def test_columns_have_unit_norm():
    S = sk.sketch_matrix(3000, 200, 8, 5)
    colnorm2 = np.asarray(S.multiply(S).sum(axis=0)).ravel()
    np.testing.assert_allclose(colnorm2, 1.0, rtol=0, atol=4e-16)
    assert S.nnz == 3000 * 8


def test_clarkson_woodruff_case():
    S = sk.sketch_matrix(1000, 50, 1, 9)
    assert S.nnz == 1000
    assert set(np.unique(S.data).tolist()) <= {-1.0, 1.0}


def test_identity_kind():
    S = sk.sketch_matrix(40, 40, 8, 1, "identity")
    assert np.array_equal(S.toarray(), np.eye(40))


def test_row_and_sign_uniformity():
    n, s, zeta = 200_000, 400, 8
    rows, signs = sk.sparse_sign_pattern(n, s, zeta, seed=11)
    counts = np.bincount(rows.ravel(), minlength=s)
    expect = n * zeta / s
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    # chi-square with s-1 dof: mean 399, sd ~28; distinctness within a column only shrinks the variance
    assert chi2 < 399 + 6 * np.sqrt(2 * 399)
    frac = float((signs > 0).mean())
    assert abs(frac - 0.5) < 6 * np.sqrt(0.25 / signs.size)


def test_subspace_embedding_distortion():
    # Eq. 1: (1-eps)||v||^2 <= ||Sv||^2 <= (1+eps)||v||^2 on a 20-dim subspace, s = 400, zeta = 8
    n, s, d = 20_000, 400, 20
    rng = np.random.default_rng(0)
    U, _ = np.linalg.qr(rng.standard_normal((n, d)))
    S = sk.sketch_matrix(n, s, 8, 21)
    sv = np.linalg.svd(S @ U, compute_uv=False)
    assert sv.max() ** 2 < 1.5 and sv.min() ** 2 > 0.5
    # mean squared norm of sketched random unit vectors is ~1 (E||Sv||^2 = ||v||^2)
    X = rng.standard_normal((n, 200))
    X /= np.linalg.norm(X, axis=0)
    assert abs(float(np.mean(np.linalg.norm(S @ X, axis=0) ** 2)) - 1.0) < 0.05
