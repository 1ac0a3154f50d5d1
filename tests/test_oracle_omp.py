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


def _splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea and Flood, 2014) on uint64 arrays."""
    x = (x + np.uint64(0x9E3779B97F4A7C15))
    x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def test_jitter_probe_moves_every_population_one_ulp(omp_lib):
    """The conditioning probe of the long-run parity bar: a jittered step is
    every population moved by one ulp, up or down as the low bit of
    SplitMix64(seed ^ step << 32, then + index) says, followed by the plain
    step.  Replayed here by hand; the OpenMP build jitters identically; a
    zero-step probe changes nothing."""
    p, phi, ux, uy = W.small_case(24, 17, seed=43)
    seed = 7
    a = oracle.Oracle(p)
    a.init_phi(phi, ux, uy)
    a.step(2)  # the probe's hash depends on the step count
    f0, g0 = a.pops()
    with np.errstate(over="ignore"):
        base = _splitmix64(np.array([seed ^ (2 << 32)], dtype=np.uint64))[0]
        n9 = f0.size
        q = np.arange(n9, dtype=np.uint64)
        df = _splitmix64(base + q) & np.uint64(1)
        dg = _splitmix64(base + np.uint64(n9) + q) & np.uint64(1)
    df, dg = df.reshape(f0.shape), dg.reshape(g0.shape)  # SoA order: slot, then cell
    fj = np.where(df == 1, np.nextafter(f0, np.inf), np.nextafter(f0, -np.inf))
    gj = np.where(dg == 1, np.nextafter(g0, np.inf), np.nextafter(g0, -np.inf))
    assert np.all(fj != f0) and np.all(gj != g0)
    a.set_pops(fj, gj)
    a.step(1)
    c = oracle.Oracle(p)
    c.init_phi(phi, ux, uy)
    c.step(2)
    c.step_jitter(1, seed)
    assert np.array_equal(a.pops()[0], c.pops()[0]) and np.array_equal(a.pops()[1], c.pops()[1])
    e = oracle.Oracle(p, lib=omp_lib)
    e.init_phi(phi, ux, uy)
    e.step(2)
    e.step_jitter(1, seed)
    assert np.array_equal(e.pops()[0], c.pops()[0]) and np.array_equal(e.pops()[1], c.pops()[1])
    z = oracle.Oracle(p)
    z.init_phi(phi, ux, uy)
    z.step(2)
    z.step_jitter(0, seed)
    assert np.array_equal(z.pops()[0], f0) and np.array_equal(z.pops()[1], g0)
