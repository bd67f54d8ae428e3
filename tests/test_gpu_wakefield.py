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


def test_far_bound_electrons_3d():
    """3D: neutral two-body ions of the medium (Z_b = 1, w_b = 3: the modified
    Coulomb field holds the bound electron with at most ~0.02) hit by an
    a0 = 3 pulse, which tears the bound electrons several cells from their
    nuclei.  Those bodies are gathered and deposited on the global grid (the
    sorted mode's far path); fields and both bodies match the oracle.  The
    atomic mode, which has no far path, reports a domain error."""
    from paper_2208_08038_gb300 import binding as B
    wl = synth.neutral_3d(seed=8, steps=60, n=(48, 16, 16), ppc=1, sigma_u=0.0, margin=3)
    wl.bc = (1, 0, 0)
    L = wl.lasers[0]
    L.a0, L.waist, L.fwhm = 3.0, 0.0, 2 * synth.T0
    L.t0 = 1.5 * L.fwhm
    ora, osid, _ = oracle_from_workload(wl)
    gpu, gsid, _ = gpu_from_workload(wl, deposit_mode=1)
    ora.step(wl.steps)
    gpu.step(wl.steps)
    gpu.sync()
    x1o, x2o, u1o, u2o = ora.bodies(osid[0])
    dist = np.linalg.norm(x1o - x2o, axis=1)
    assert dist.max() > 3 * wl.dx[0], dist.max()  # the far path ran
    err = field_rel_l2(gpu.fields(), ora.fields())
    print(f"far bodies 3D: {int((dist > wl.dx[0]).sum())} ions with r > dx, E,B rel L2 {err:.3e}")
    assert err < 1e-3, err
    x1g, x2g, u1g, u2g = gpu.read_particles(gsid[0], len(x1o))
    Lb = np.array(wl.n) * np.array(wl.dx)
    d = (x2g - x2o + 0.5 * Lb) % Lb - 0.5 * Lb
    assert np.abs(d).max() < 1e-3 * wl.dx[0], np.abs(d).max()
    assert rel_l2(u2g, u2o) < 1e-3
    gpu.close()
    ora.close()
    # the atomic mode has no far path: a domain error
    gpu, _, _ = gpu_from_workload(wl, deposit_mode=0)
    gpu.step(wl.steps)
    with pytest.raises(B.BPError) as e:
        gpu.sync()
    assert e.value.code == B.BP_ERR_DOMAIN
    gpu.close()
