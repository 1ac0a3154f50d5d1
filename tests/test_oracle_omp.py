"""The OpenMP build of the oracle (same source, liborc_omp.so) against the
serial build: every pass it parallelises writes disjoint cells with the
same per-cell arithmetic, so the states must agree bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1507_03521_gb300 import workloads as W


@pytest.fixture(scope="module")
def omp_lib():
    try:
        path = oracle.build_omp()
    except Exception as e:  # no OpenMP in this toolchain
        pytest.skip(f"OpenMP build unavailable: {e}")
    assert oracle.set_threads(4, path) == 4
    return path


@pytest.mark.parametrize("walls", [False, True])
def test_omp_build_is_bit_identical(omp_lib, walls):
    p, phi, ux, uy = W.small_case(40, 33, seed=41, walls=walls, gravity=1e-5 if walls else 0.0,
                                  u_wall=0.01 if walls else 0.0)
    a = oracle.Oracle(p)
    b = oracle.Oracle(p, lib=omp_lib)
    for o in (a, b):
        o.init_phi(phi, ux, uy)
        o.step(25)
    fa, ga = a.pops()
    fb, gb = b.pops()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert a.mass() == b.mass()
    for k, v in a.fields().items():
        assert np.array_equal(v, b.fields()[k]), k
