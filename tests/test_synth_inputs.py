"""The seeded input generators produce what the input recipe states (CPU only).

- SplitMix64 matches its published reference outputs, and the uniforms / normals have the
  expected moments.
- The Gaussian test matrix Omega (Def. 2) has four iid N(0, 1) planes, or only the real plane
  with real_only.
- Constructed spectra (config 1 style) have exactly the requested singular values.
- The completion inputs are pure, of exact rank r, with the requested share of removed entries;
  the random low-rank example has rank exactly 50.
"""
import numpy as np

import synth
from oracle.qsvd import singular_values


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 1234567: the first outputs of the published reference implementation
    # (state += 0x9E3779B97F4A7C15, then the two xor-shift-multiply rounds).
    got = synth.splitmix64(1234567, np.arange(3, dtype=np.uint64))
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423]
    assert [int(x) for x in got] == want


def test_uniform_and_gaussian_moments():
    u = synth.uniform(7, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    g = synth.gaussian(8, 200000)
    assert abs(g.mean()) < 1e-2 and abs(g.var() - 1.0) < 2e-2
    assert abs((g ** 4).mean() - 3.0) < 0.1


def test_omega_planes():
    om = synth.gaussian_qmat(9, 300, 40)
    assert om.shape == (4, 300, 40)
    for c in range(4):
        assert abs(om[c].std() - 1.0) < 0.05
    r = synth.gaussian_qmat(9, 300, 40, real_only=True)
    assert np.all(r[1:] == 0.0) and abs(r[0].std() - 1.0) < 0.05


def test_constructed_spectrum():
    sig = np.zeros(40)
    sig[:10] = 0.5 ** np.arange(10)
    A = synth.spectrum_matrix(60, 40, sig, seed=3)
    s = singular_values(A)
    np.testing.assert_allclose(s[:10], sig[:10], rtol=1e-12)
    assert s[10:].max() < 1e-13


def test_completion_inputs():
    P = synth.completion_problem(90, 70, 6, missing=0.7, seed=4)
    assert np.all(P.A[0] == 0.0) and P.pure
    s = singular_values(P.A)
    assert s[5] > 1e-3 * s[0] and s[6] < 1e-12 * s[0]
    mask = P.extra["mask"]
    assert mask.dtype == np.uint8 and set(np.unique(mask)) <= {0, 1}
    assert abs(mask.mean() - 0.3) < 0.03
    assert abs(np.sqrt((P.A[1:] ** 2).mean()) - 1.0) < 1e-12
    assert P.Omega.shape == (4, 70, P.k + P.p)


def test_random_lowrank_example_has_rank_50():
    P = synth.random_lowrank_problem(200, 180, 50)
    s = singular_values(P.A)
    assert s[49] > 1e-6 * s[0] and s[50] < 1e-12 * s[0]
    assert P.k == 50 and P.Omega.shape == (4, 180, 60)
