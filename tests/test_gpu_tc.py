"""The tensor-core (tcgen05, TF32) spatial transforms of the preconditioner
agree with the CUDA-core transforms on a ragged problem."""

import pytest

from tests.gpu_helpers import library

pytestmark = pytest.mark.gpu


def test_tc_transform_selftest():
    P = library()
    from paper_2311_17500_gb300._lib import tc_selftest
    usable, err = tc_selftest()
    # TF32 inputs: 11-bit significands (unit roundoff 2^-11), 131-term sums
    assert usable, f"tensor-core transform self-test failed, max rel err {err}"
    assert err < 5e-3
