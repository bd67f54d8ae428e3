"""GPU run of the x-ray wakefield application (Sec. 3.2: the pre-ionised
gold crystal, 30 free electrons per ion, driven at a0 = 3) against the FP64
oracle on 256 x 64 cells of the configuration: relative field L2 <= 1e-5
after one step and <= 1e-3 after 300 steps, once the pulse is inside the
crystal.  The run is in the regime it is meant to exercise: the free
electrons' quiver is relativistic (max |u| > 1.5) and the bound electrons of
the two-body ions are torn far beyond a_c (into the Coulomb tail of the
modified potential).  Gauss's law holds through the run."""
import numpy as np
import pytest

from paper_2208_08038_gb300 import synth
from _common import field_rel_l2, gpu_from_workload, oracle_from_workload, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"


def reduced():
    wl = synth.wakefield_2d(n=(256, 64), span=(2.0, 6.0), steps=300)
    wl.lasers[0].fwhm = 2 * synth.T0
    wl.lasers[0].t0 = 1.5 * wl.lasers[0].fwhm
    return wl


def test_wakefield_reduced_parity_and_regime():
    wl = reduced()
    ora, osid, _ = oracle_from_workload(wl)
    gpu, gsid, _ = gpu_from_workload(wl, deposit_mode=1)
    R0 = gpu.residual()
    ora.step(1)
    gpu.step(1)
    gpu.sync()
    assert field_rel_l2(gpu.fields(), ora.fields()) < 1e-5
    ora.step(wl.steps - 1)
    gpu.step(wl.steps - 1)
    gpu.sync()
    err = field_rel_l2(gpu.fields(), ora.fields())
    print(f"wakefield: E,B rel L2 {err:.3e} after {wl.steps} steps")
    assert err < 1e-3, err
    # the regime
    _, _, ue, _ = ora.bodies(osid[1])
    assert np.sqrt((ue ** 2).sum(axis=1)).max() > 1.5
    x1, x2, _, _ = ora.bodies(osid[0])
    assert np.linalg.norm(x1 - x2, axis=1).max() > 10 * ora.ac(osid[0], 0)
    # charge conservation (off the open x faces and the antenna plane)
    R = gpu.residual()
    keep = np.ones(wl.n[0], dtype=bool)
    keep[:3] = keep[-3:] = False
    keep[wl.lasers[0].ia - 2:wl.lasers[0].ia + 3] = False
    qe = max(abs(sp.w * (sp.q if isinstance(sp, synth.Free) else sp.Zb)) for sp in wl.species)
    assert np.abs((R - R0)[..., keep]).max() < 1e-3 * qe
    gpu.close()
    ora.close()
