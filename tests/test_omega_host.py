"""The library's seeded test matrix (Def. 2) on the host: qlr_gaussian_qmat_host draws the same
Gaussian quaternion matrix as the seeded input module that the tests and the oracle use, from the
published SplitMix64 and Box-Muller definitions written independently on each side.  No GPU."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def qlr():
    from paper_2507_13731_gb300 import build
    build.build()
    from paper_2507_13731_gb300 import qlr as q
    return q


def test_splitmix64_matches_the_input_module(qlr):
    for seed in (0, 1234567, 2 ** 63 + 5):
        for t in (0, 1, 2, 99):
            assert qlr.splitmix64(seed, t) == int(synth.splitmix64(seed, np.array([t], dtype=np.uint64))[0])
    # the workloads' test matrices use the stream seed of tag 6 (TAG_OMEGA)
    assert qlr.splitmix64(1235, synth.TAG_OMEGA) == synth.stream_seed(1235, synth.TAG_OMEGA)


@pytest.mark.parametrize("rows,cols,real_only", [(7, 3, False), (192, 15, False), (33, 5, True), (1, 1, False)])
def test_gaussian_qmat_matches_the_input_module(qlr, rows, cols, real_only):
    seed = synth.stream_seed(1234, synth.TAG_OMEGA)
    got = qlr.gaussian_qmat_host(seed, rows, cols, real_only).numpy()
    want = synth.gaussian_qmat(seed, rows, cols, real_only=real_only)
    # the two sides evaluate log / cos / sin with different libraries: agreement to a few ulp
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    if real_only:
        assert np.all(got[1:] == 0.0)


def test_config1_omega_from_the_seed(qlr):
    P = synth.config1()
    got = qlr.gaussian_qmat_host(qlr.splitmix64(1234, synth.TAG_OMEGA), P.n, P.ell).numpy()
    np.testing.assert_allclose(got, P.Omega, rtol=1e-13, atol=1e-13)


def test_host_generator_rejects_bad_arguments(qlr):
    L = qlr.lib()
    assert L.qlr_gaussian_qmat_host(1, 3, 3, 0, None) == qlr.EINVAL
    assert L.qlr_gaussian_qmat_host(1, -1, 3, 0, 1) == qlr.EINVAL
