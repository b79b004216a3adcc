"""Failure detection on the GPU without a fault.

The wavefront kernels wait on their neighbour tiles, and every such wait is
bounded by elapsed time.  Here one tile is told never to report its sweep
(pcad_chain_inject_stall), so the tiles around it wait for a dependency that
never arrives.  With a 5 ms limit the launch must end promptly, the chain
must report PCAD_ETIMEOUT, and the context must stay usable: after the stall
is removed and the chain reset, the same run reproduces the oracle.  Nothing
here traps, faults or hangs the GPU: the waits give up by design."""
import time

import numpy as np
import pytest

import oracle
from pcad_inputs import Model, gaussian_noise, greyscale_scene

pytestmark = pytest.mark.gpu

ETIMEOUT = 4


@pytest.fixture(scope="module")
def pc():
    import paper_2507_14869_gb300 as pc
    pc.lib()
    return pc


def _case(L, sigma, H=64, W=256, seed=31):
    clean = greyscale_scene(seed, H, W, L, n_shapes=6)
    return gaussian_noise(seed + 1, clean, sigma, L)


CASES = {
    # CUDA-core wavefront: 16 x 8 tiles of 4 x 32 sites
    "wave_L16": (16, 1.0, dict(pair_coef=0.6, pair_T=3, inertia=1.5), 3),
    # tensor-core wavefront, lazy PCA and checkerboard Gibbs
    "tensor_L256": (256, 20.0, dict(pair_coef=0.05, pair_T=30, inertia=2.0), 2),
    "tensor_gibbs_L256": (256, 20.0, dict(pair_coef=0.05, pair_T=30, sampler=1), 2),
    # windowed CUDA-core wavefronts: 4 x 32 tiles (PCA), 4 x 64 cell tiles (Gibbs)
    "window_wave_L256": (256, 20.0, dict(pair_coef=0.05, pair_T=30, inertia=2.0), 7),
    "window_wave_gibbs_L256": (256, 20.0, dict(pair_coef=0.05, pair_T=30, sampler=1), 7),
}


@pytest.mark.parametrize("name", list(CASES))
def test_lost_dependency_times_out_promptly(pc, name):
    L, sigma, kw, kind = CASES[name]
    g = _case(L, sigma)
    m = Model(L=L, pair=1, sigma=sigma, **kw)
    sampler = kw.get("sampler", 0)
    with pc.Chain(g, m, seed=5, chain_id=7, burn_in=8) as ch:
        ch.set_kernel(kind)
        assert ch.kernel_in_use() == kind
        ch.run(32)            # a healthy run first: graphs built, kernel attributes set
        ch.sync()
        x_ok = ch.sample()
        ch.set_wait_limit(0.005).inject_stall(45).reset()
        t0 = time.perf_counter()
        ch.run(32)
        with pytest.raises(pc.PcadError) as e:
            ch.sync()
        dt = time.perf_counter() - t0
        assert e.value.status == ETIMEOUT
        assert dt < 1.0, f"the stalled launch took {dt:.3f} s to end"
        # the context is still usable: stall off, reset, same result as before
        ch.inject_stall(-1).reset()
        ch.run(32)
        ch.sync()
        assert np.array_equal(ch.sample(), x_ok)
    kwo = {} if sampler == 0 else {"order": oracle.ORDER_COLOUR}
    xo, _, _, _ = oracle.run_chain(m, g, 32, 8, seed=5, chain=7, sampler=sampler, **kwo)
    assert np.array_equal(x_ok, xo)


def test_wait_limit_and_stall_are_validated(pc):
    g = _case(16, 1.0, H=8, W=64)
    m = Model(L=16, pair=1, pair_coef=0.6, pair_T=3, sigma=1.0, inertia=1.0)
    with pc.Chain(g, m, seed=1) as ch:
        for bad in (0.0, -1.0, 1e-5, 61.0, float("nan")):
            with pytest.raises(pc.PcadError) as e:
                ch.set_wait_limit(bad)
            assert e.value.status == 1
        for bad in (-2, 4, 1000):      # 8 x 64 holds 2 x 2 tiles
            with pytest.raises(pc.PcadError) as e:
                ch.inject_stall(bad)
            assert e.value.status == 1
        ch.set_wait_limit(2.0).inject_stall(3).inject_stall(-1)
