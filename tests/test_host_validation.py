"""Host-side validation of the C ABI, run without a GPU: every rejection below
happens before any CUDA call, with SIM_EINVAL and a message naming the cause."""
import numpy as np
import pytest

import paper_2303_00689_gb300 as kx
import synth


def _create(cfg=None, Z=None, R=None, charge=0):
    mol = synth.c4h6(1)
    cfg = cfg or kx.sim_config_default()
    table = kx.param_table(synth.table_to_array(synth.synthetic_table(1)))
    return kx.sim_create(cfg, table, mol.Z if Z is None else Z, mol.R if R is None else R, charge=charge)


@pytest.mark.parametrize("field,value", [("Te", 0.0), ("dt", -0.5), ("m_max", 0), ("m_max", 17),
                                         ("m_min", 9), ("scf_mix", 1.0), ("scf_max", 0), ("kernel", 7),
                                         ("xl_c", float("nan")), ("langevin_gamma", -1.0),
                                         ("langevin_T", float("inf")), ("precision", 5)])
def test_invalid_configuration_is_rejected(field, value):
    cfg = kx.sim_config_default(m_max=4, m_min=4)
    setattr(cfg, field, value)
    with pytest.raises(kx.SimError) as e:
        _create(cfg)
    assert e.value.code == kx.SIM_EINVAL


def test_unsupported_element_and_odd_electron_count_are_rejected():
    mol = synth.c4h6(1)
    Z = mol.Z.copy()
    Z[0] = 9
    with pytest.raises(kx.SimError) as e:
        _create(Z=Z)
    assert e.value.code == kx.SIM_EINVAL and "atomic number" in str(e.value)
    with pytest.raises(kx.SimError) as e:
        _create(charge=1)
    assert e.value.code == kx.SIM_EINVAL and "electron" in str(e.value)
    R = mol.R.copy()
    R[2, 0] = np.inf
    with pytest.raises(kx.SimError) as e:
        _create(R=R)
    assert e.value.code == kx.SIM_EINVAL


def test_batch_and_server_arguments_are_checked():
    with pytest.raises(kx.SimError) as e:
        kx.sim_batch_step([None], 1)
    assert e.value.code == kx.SIM_EINVAL
    with pytest.raises(kx.SimError) as e:
        kx.sim_batch_create([])
    assert e.value.code == kx.SIM_EINVAL
    assert kx.lib().sim_server_create(None, None) == kx.SIM_EINVAL
