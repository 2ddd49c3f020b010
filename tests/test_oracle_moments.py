"""The oracle's beam moments (oracle.track.moments_vector, FP64 two-pass, and
moments_vector_exact, rational arithmetic) pinned by closed forms, hand-worked
tiny bunches and invariants of the definition mean_a = sum x_a / N,
C_ab = sum (x_a - mean_a)(x_b - mean_b) / N."""
import numpy as np
import pytest

from oracle import track as tr

IU = np.triu_indices(6)


def _pair_index(a, b):
    return 6 + [k for k, (i, j) in enumerate(zip(*IU)) if i == a and j == b][0]


def test_hand_worked_three_particles():
    # x = (1, 2, 6): mean 3, variance ((-2)^2 + (-1)^2 + 3^2) / 3 = 14/3;
    # px = (0, 0, 3): mean 1, C_x,px = ((-2)(-1) + (-1)(-1) + 3*2) / 3 = 3
    c = np.zeros((6, 3))
    c[0] = [1.0, 2.0, 6.0]
    c[1] = [0.0, 0.0, 3.0]
    for f in (tr.moments_vector, tr.moments_vector_exact):
        m = f(c)
        assert m[0] == pytest.approx(3.0, rel=1e-15) and m[1] == pytest.approx(1.0, rel=1e-15)
        assert m[_pair_index(0, 0)] == pytest.approx(14.0 / 3.0, rel=1e-15)
        assert m[_pair_index(0, 1)] == pytest.approx(3.0, rel=1e-15)
        assert m[_pair_index(1, 1)] == pytest.approx(2.0, rel=1e-15)   # (1 + 1 + 4) / 3


def test_symmetric_pairs_closed_form():
    # two particles mu -/+ a per coordinate, with signs s_a: mean mu, C_ab = s_a s_b a_a a_b
    mu = np.array([1e-3, -2e-4, 3e-3, 0.0, 5e2, -1e-5])
    amp = np.array([2.0 ** -12, 2.0 ** -20, 2.0 ** -9, 2.0 ** -30, 2.0 ** -3, 2.0 ** -25])
    sg = np.array([1, -1, 1, 1, -1, 1])
    c = np.stack([mu - sg * amp, mu + sg * amp], axis=1)
    m = tr.moments_vector_exact(c)
    for a in range(6):
        assert m[a] == pytest.approx(mu[a], rel=1e-15, abs=0)
        for b in range(a, 6):
            assert m[_pair_index(a, b)] == pytest.approx(sg[a] * sg[b] * amp[a] * amp[b],
                                                         rel=1e-15)


def test_constant_coordinate_has_its_value_and_no_spread():
    rng = np.random.default_rng(1)
    c = rng.normal(size=(6, 101))
    c[3] = 1e-3                                    # every particle the same
    m = tr.moments_vector_exact(c)
    assert m[3] == 1e-3
    for b in range(6):
        a, bb = min(3, b), max(3, b)
        assert m[_pair_index(a, bb)] == 0.0


def test_exact_and_fp64_agree_and_order_is_irrelevant():
    rng = np.random.default_rng(4)
    c = rng.normal(size=(6, 2_001)) * np.array([1e-3, 1e-4, 2e-3, 3e-4, 1e-2, 1e-5])[:, None]
    c[4] += 3.0                                    # an offset coordinate
    ex = tr.moments_vector_exact(c)
    fp = tr.moments_vector(c)
    assert np.abs(ex - fp).max() <= 1e-14 * np.abs(ex).max()
    perm = rng.permutation(c.shape[1])
    assert np.array_equal(tr.moments_vector_exact(c[:, perm]), ex)


def test_translation_moves_the_means_only():
    rng = np.random.default_rng(5)
    c = np.round(rng.normal(size=(6, 301)) * 2 ** 20) * 2.0 ** -30   # dyadic: shifts are exact
    shift = np.array([0.5, -0.25, 1.0, 2.0, -8.0, 0.125])
    m0 = tr.moments_vector_exact(c)
    m1 = tr.moments_vector_exact(c + shift[:, None])
    assert np.array_equal(m1[6:], m0[6:])
    assert np.allclose(m1[:6], m0[:6] + shift, rtol=0, atol=1e-15)
