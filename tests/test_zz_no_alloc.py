"""The allocation-free PCG entry point (bdem_pcg_static) against the allocating one (bdem_debug_pcg).

bdem_pcg_static is for callers that cannot allocate device memory (an external pool that forbids cudaMalloc,
or a thread that must not allocate while other work is being captured): its scratch lives in a static device
array of the library. Both calls run the block-Jacobi PCG without FP64-residual refinement here (pcg_refine = 0),
so they solve the same way. This file is collected last so that a run stopping at the first failure has already run
every other test; test_in_a_fresh_process runs the comparison again in a new Python process, where the static
array's first use (the symbol lookup) happens in that process.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2308_10459_gb300 as pkg
from paper_2308_10459_gb300 import build as bmod
from paper_2308_10459_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bmod.build()
    pkg.load()
    return torch


def assembled_sim(prec, kinematic=False):
    """A deformed 3x3x3 contact lattice with its Newton system assembled; with kinematic=True its bottom layer is
    kinematic (those rows leave the solve)."""
    from scipy.spatial.transform import Rotation
    sc = scenes.cube_lattice(nx=3, spacing=0.0098, r=0.005, k_ground=1e6, z_bottom=0.0045, k_self=1e5,
                             contact_skin=0.005)
    if kinematic:
        sc.kinematic[sc.pos[:, 2] < sc.pos[:, 2].min() + 1e-6] = 1
    rng = np.random.default_rng(4)
    p = sc.pos + rng.normal(size=sc.pos.shape) * 3e-4
    q = Rotation.from_rotvec(rng.normal(size=(sc.n, 3)) * 0.2).as_quat()
    sim = pkg.Sim(sc, precision=prec, config=dict(pcg_refine=0))
    sim.write_state(p, q, rng.normal(size=(sc.n, 3)) * 0.1, rng.normal(size=(sc.n, 4)) * 0.1)
    sim.bdem_debug_system(p + 1e-4, q + 0.01, want_bonds=False)
    return sim, sc


@pytest.mark.parametrize("kinematic", [False, True], ids=["free", "kinematic-layer"])
@pytest.mark.parametrize("prec,eps,tol", [(pkg.BDEM_FP64, 1e-12, 1e-8), (pkg.BDEM_MIXED, 1e-6, 1e-3)])
def test_static_pcg_matches_allocating_pcg_twice(torch_cuda, prec, eps, tol, kinematic):
    """Two calls in a row give the allocating solve's answer, and neither changes the device's free memory."""
    torch = torch_cuda
    sim, sc = assembled_sim(prec, kinematic)
    b = np.random.default_rng(6).normal(size=(sc.n, 6))
    kin = sc.kinematic.astype(bool)
    b[kin] = 0.0
    x_ref, it_ref = sim.bdem_debug_pcg(b, eps, 2000)
    b_dev = torch.tensor(b, dtype=torch.float64, device="cuda")
    x_devs = [torch.full((sc.n, 6), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    sim.bdem_pcg_static(b_dev.data_ptr(), x_devs[2].data_ptr(), eps, 2000)  # first use: the symbol lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(2):
        it = sim.bdem_pcg_static(b_dev.data_ptr(), x_devs[call].data_ptr(), eps, 2000)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, call  # the call allocated nothing
        x = x_devs[call].cpu().numpy()
        assert np.abs(x - x_ref).max() <= tol * np.abs(x_ref).max(), call
        assert abs(int(it[0]) - int(it_ref[0])) <= 2, call
        if kinematic:
            assert np.all(x[kin] == 0.0), call
    sim.close()


def test_in_a_fresh_process(torch_cuda):
    """The comparison above, alone in a new Python process."""
    if os.environ.get("BDEM_NO_ALLOC_CHILD"):
        pytest.skip("already the child process")
    env = dict(os.environ, BDEM_NO_ALLOC_CHILD="1")
    out = subprocess.run([sys.executable, "-m", "pytest", os.path.abspath(__file__), "-q", "-m", "gpu", "-p",
                          "no:cacheprovider", "-k", "matches_allocating"], capture_output=True, text=True,
                         timeout=600, env=env, cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-2000:]
    assert " passed" in out.stdout and "failed" not in out.stdout


def test_static_pcg_rejects_systems_beyond_its_array(torch_cuda):
    torch = torch_cuda
    n = 300_000  # more than the 24 MiB array holds in either precision
    pos = np.stack([np.arange(n) * 0.01, np.zeros(n), np.ones(n)], 1)
    sc = scenes._assemble(pos, np.full(n, 0.004), np.zeros(n, np.int32), np.zeros(n, np.uint8),
                          np.zeros((0, 2), np.int64), [scenes.Material(1e7, 0.3, 2500.0)],
                          scenes.default_config(), "line")
    sim = pkg.Sim(sc, precision=pkg.BDEM_MIXED)
    b = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.BdemError) as ei:
        sim.bdem_pcg_static(b.data_ptr(), b.data_ptr(), 1e-6, 10)
    assert ei.value.status == pkg.BDEM_E_INVALID and "static PCG scratch" in str(ei.value)
    sim.close()
