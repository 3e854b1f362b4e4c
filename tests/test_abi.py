"""The C-ABI library builds, loads, and exports every function include/sim.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2303_00689_gb300 as kx
from paper_2303_00689_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def _declared():
    names = set()
    for f in os.listdir(HEADER):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(HEADER, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\*\s]+?\b(sim_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def library():
    build.build()
    return ctypes.CDLL(kx.LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sim_create", "sim_step", "sim_get_state", "sim_destroy", "sim_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(library):
    missing = [n for n in sorted(_declared()) if not hasattr(library, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_names_match_header():
    assert set(kx.EXPORTED) <= _declared()


def test_config_defaults_without_gpu(library):
    cfg = kx.sim_config_default()
    assert cfg.Te == 1000.0 and cfg.dt == 0.5 and cfg.m_max == 4 and cfg.scf_mix == 0.1


def test_load_rejects_files_that_are_not_checkpoints(tmp_path):
    """sim_load validates the whole file before touching a device."""
    import paper_2303_00689_gb300 as kx
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"not a checkpoint at all")
    for path in (bad, tmp_path / "missing.ckpt"):
        with pytest.raises(kx.SimError) as e:
            kx.sim_load(str(path))
        assert e.value.code == kx.SIM_EINVAL


def test_memory_estimate_is_host_arithmetic():
    """sim_estimate_bytes (used by the server's HBM-budget admission) needs no
    device: it grows with the basis, the mixed path adds its BF16 slice slots,
    and invalid input gives 0."""
    import numpy as np
    import paper_2303_00689_gb300 as kx
    small = np.array([6, 6, 1, 1], dtype=np.int32)
    big = np.array([6] * 40 + [1] * 20, dtype=np.int32)
    c64 = kx.sim_config_default(m_max=4, m_min=4)
    cmx = kx.sim_config_default(m_max=4, m_min=4, precision=kx.SIM_PREC_MIXED)
    assert 0 < kx.sim_estimate_bytes(c64, small) < kx.sim_estimate_bytes(c64, big)
    assert kx.sim_estimate_bytes(cmx, big) > kx.sim_estimate_bytes(c64, big)
    n = 40 * 4 + 20
    # at least the ~30 n x n FP64 matrices of the layout
    assert kx.sim_estimate_bytes(c64, big) > 30 * n * n * 8
    bad = kx.sim_config_default(m_max=0)
    assert kx.sim_estimate_bytes(bad, big) == 0
