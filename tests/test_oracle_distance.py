"""Pins for the oracle's canonical distance (Section 2: Euclidean distance on
float32 vectors, angular data L2-normalised; uint8 byte vectors).

The canonical float32 summation order is a reading (the paper fixes none); it
is pinned here by what does not depend on the order: exact results on
integer-valued inputs, the gamma_n rounding bound against float64 (Higham,
Accuracy and Stability of Numerical Algorithms, Sec. 3.1), exact uint8
arithmetic and symmetry.
"""
import numpy as np
import pytest

import oracle

U = 2.0 ** -24


def _pair_data(rng, n, d, kind):
    if kind == "int":
        X = rng.integers(-8, 9, size=(n, d)).astype(np.float32)
    else:
        X = rng.normal(size=(n, d)).astype(np.float32)
    return X


@pytest.mark.parametrize("d", [1, 3, 4, 16, 100, 128, 129, 300, 960])
def test_l2_exact_on_integers(d):
    rng = np.random.default_rng(d)
    X = _pair_data(rng, 6, d, "int")
    D = oracle.Data(X, d, oracle.L2_F32)
    for i in range(6):
        for j in range(6):
            exact = int(((X[i].astype(np.int64) - X[j].astype(np.int64)) ** 2).sum())
            assert oracle.dist(D, i, j) == float(exact)


@pytest.mark.parametrize("d", [4, 16, 100, 128, 960])
def test_angular_exact_on_integers(d):
    rng = np.random.default_rng(100 + d)
    X = rng.integers(-3, 4, size=(5, d)).astype(np.float32)
    D = oracle.Data(X, d, oracle.ANGULAR_F32)
    for i in range(5):
        for j in range(5):
            dot = int((X[i].astype(np.int64) * X[j].astype(np.int64)).sum())
            assert oracle.dist(D, i, j) == np.float32(1.0) - np.float32(dot)


@pytest.mark.parametrize("d", [16, 100, 128, 257, 960])
def test_l2_within_rounding_bound(d):
    rng = np.random.default_rng(7 + d)
    X = _pair_data(rng, 12, d, "float")
    D = oracle.Data(X, d, oracle.L2_F32)
    g = (d + 8) * U / (1 - (d + 8) * U)
    for i in range(12):
        for j in range(12):
            ref = oracle.dist_f64(D, i, j)
            x64 = X[i].astype(np.float64) - X[j].astype(np.float64)
            assert ref == pytest.approx(float((x64 * x64).sum()), rel=1e-12, abs=1e-300)
            assert abs(oracle.dist(D, i, j) - ref) <= g * ref


@pytest.mark.parametrize("d", [16, 100, 960])
def test_angular_within_rounding_bound(d):
    rng = np.random.default_rng(11 + d)
    X = rng.normal(size=(10, d))
    X = (X / np.linalg.norm(X, axis=1, keepdims=True)).astype(np.float32)
    D = oracle.Data(X, d, oracle.ANGULAR_F32)
    g = (d + 8) * U / (1 - (d + 8) * U)
    for i in range(10):
        for j in range(10):
            absdot = float(np.abs(X[i].astype(np.float64) * X[j].astype(np.float64)).sum())
            ref = oracle.dist_f64(D, i, j)
            # dot error <= gamma * sum|x y|; the final 1 - dot adds one rounding
            assert abs(oracle.dist(D, i, j) - ref) <= g * absdot + 2 * U * (1 + abs(ref))


@pytest.mark.parametrize("d", [1, 16, 128, 256])
def test_uint8_exact(d):
    rng = np.random.default_rng(d)
    X = rng.integers(0, 256, size=(8, d)).astype(np.uint8)
    D = oracle.Data(X, d, oracle.L2_U8)
    for i in range(8):
        for j in range(8):
            exact = int(((X[i].astype(np.int64) - X[j].astype(np.int64)) ** 2).sum())
            assert oracle.dist(D, i, j) == float(exact)


def test_symmetric_bitwise():
    rng = np.random.default_rng(3)
    for metric in (oracle.L2_F32, oracle.ANGULAR_F32):
        X = rng.normal(size=(9, 100)).astype(np.float32)
        D = oracle.Data(X, 100, metric)
        for i in range(9):
            for j in range(9):
                a, b = oracle.dist(D, i, j), oracle.dist(D, j, i)
                assert np.float32(a).tobytes() == np.float32(b).tobytes()


def test_padding_beyond_d_is_ignored():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(4, 20)).astype(np.float32)
    Xp = np.zeros((4, 24), np.float32)
    Xp[:, :20] = X
    Xg = Xp.copy()
    Xg[:, 20:] = 99.0  # garbage in the padding must not matter
    D1 = oracle.Data(Xp, 20, oracle.L2_F32)
    D2 = oracle.Data(Xg, 20, oracle.L2_F32)
    for i in range(4):
        for j in range(4):
            assert oracle.dist(D1, i, j) == oracle.dist(D2, i, j)


def test_self_distance_zero():
    rng = np.random.default_rng(9)
    X = rng.normal(size=(5, 100)).astype(np.float32)
    D = oracle.Data(X, 100, oracle.L2_F32)
    for i in range(5):
        assert oracle.dist(D, i, i) == 0.0


def test_roots_distinct_and_keyed():
    r1 = oracle.roots(0, 8, 1000)
    r2 = oracle.roots(0, 8, 1000)
    r3 = oracle.roots(1, 8, 1000)
    assert (r1 == r2).all()
    assert len(set(r1.tolist())) == 8
    assert (r1 != r3).any()
    assert ((r1 >= 0) & (r1 < 1000)).all()
    # T == n forces the collision rule to enumerate every id
    assert sorted(oracle.roots(5, 7, 7).tolist()) == list(range(7))


def test_splitmix64_is_a_bijective_mixer():
    # SplitMix64's output function is a bijection of 64-bit words (two
    # xorshift-multiply rounds with odd multipliers and a final xorshift);
    # distinct states must give distinct outputs, and state 0 maps to the
    # finaliser of the golden-ratio increment, which is nonzero.
    outs = {oracle.splitmix64(z) for z in range(4096)}
    assert len(outs) == 4096
    assert oracle.splitmix64(0) != 0


def test_splitmix64_reference_outputs():
    # The reference sequence of SplitMix64 (Steele, Lea and Flood, OOPSLA
    # 2014) seeded with 0: its first two outputs are 0xE220A8397B1DCDAF and
    # 0x6E789E6AA1B965F4.  The generator advances its state by the
    # golden-ratio increment before mixing, so the second output is the first
    # output of the generator started at that increment.  A wrong constant,
    # shift or multiplier changes both.
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
