"""The C-ABI library loads without a GPU and exports every entry point that
include/*.h declares; host-side argument validation works without a GPU.
CPU only."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(pcad_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def so():
    from paper_2507_14869_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("pcad_chain_create", "pcad_chain_run", "pcad_chain_read_sample",
                     "pcad_chain_read_mean", "pcad_metrics", "pcad_chain_export",
                     "pcad_chain_import", "pcad_chain_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(so):
    lib = ctypes.CDLL(so)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_exports_are_c_symbols_and_no_oracle_code(so):
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in declared_functions():
        assert n in syms, n                      # unmangled (extern "C")
    assert not any(s.startswith("orc_") for s in syms)


def test_binding_has_same_names(so):
    import paper_2507_14869_gb300 as pc
    for n in declared_functions():
        assert hasattr(pc, n), n


def test_host_validation_without_gpu(so):
    """Parameter checks run before any CUDA call, so they work on a CPU machine."""
    import paper_2507_14869_gb300 as pc
    g = np.zeros((4, 4), dtype=np.uint8)
    base = dict(L=16, nbhd=4, pair=1, pair_coef=0.05, pair_T=30, noise=0, sigma=2.0,
                flip_p=0.1, inertia=1.0, sampler=0)
    bad = [dict(L=1), dict(L=300), dict(nbhd=5), dict(pair_coef=float("nan")),
           dict(pair_T=300), dict(pair_coef=1.0), dict(sigma=-1.0), dict(noise=1),
           dict(inertia=50.0), dict(sampler=7)]
    for upd in bad:
        m = dict(base, **upd)
        with pytest.raises(pc.PcadError) as e:
            pc.pcad_chain_create(g, m, seed=1)
        assert e.value.status == 1, upd
    with pytest.raises(pc.PcadError):
        pc.pcad_chain_create(g, base, seed=1, chain_id=1 << 24)
    with pytest.raises(pc.PcadError):
        pc.pcad_chain_create(g, base, seed=1, burn_in=-1)
    assert pc.pcad_status_str(0) == "ok"
    assert "sm_103a" in pc.pcad_version()


def test_batch_rejects_observations_outside_the_labels_without_gpu(so):
    """Batch and server jobs are checked as chains are: an observed value
    >= L is refused (PCAD_EINVAL) before any CUDA call."""
    import paper_2507_14869_gb300 as pc
    m2 = dict(L=2, nbhd=4, pair=0, pair_coef=1.2, pair_T=1, noise=1, sigma=1.0, flip_p=0.1,
              inertia=1.0, sampler=0)
    m16 = dict(L=16, nbhd=4, pair=1, pair_coef=0.05, pair_T=30, noise=0, sigma=1.0,
               flip_p=0.1, inertia=2.0, sampler=0)
    for m, bad_value in ((m2, 2), (m16, 16), (m16, 255)):
        g = np.zeros((5, 7), dtype=np.uint8)
        g[4, 6] = bad_value   # the last site, to reach the end of the scan
        with pytest.raises(pc.PcadError) as e:
            pc.pcad_batch_create([(g, m, 1, 0, 0)], autotune=False)
        assert e.value.status == 1
        assert "observed labels" in str(e.value)
