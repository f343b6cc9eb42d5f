"""The device-memory hook of bdem_config (bdem_allocator): a simulation whose buffers come from PyTorch's caching
allocator steps bit-identically to one that uses cudaMalloc, takes every buffer from the hook while it lives, and
returns all of them at bdem_destroy."""
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


@pytest.mark.parametrize("prec", [pkg.BDEM_FP64, pkg.BDEM_MIXED], ids=["fp64", "mixed"])
def test_torch_allocator_hook(torch_cuda, prec):
    torch = torch_cuda
    sc = scenes.c2_plate_small(R=0.012)  # ground and self contact: the contact arrays grow during the steps
    ref = pkg.Sim(sc, precision=prec)
    ref.step(3)
    want = ref.read_state()
    ref.close()
    hook = pkg.TorchAllocator()
    before = torch.cuda.memory_allocated()
    sim = pkg.Sim(sc, precision=prec, allocator=hook)
    sim.step(3)
    got = sim.read_state()
    assert hook.calls > 10 and len(hook.live) > 10
    assert torch.cuda.memory_allocated() - before >= sum(hook.live.values())
    for k in ("pos", "quat", "vel", "quat_vel", "broken"):
        assert np.array_equal(got[k], want[k]), k
    sim.close()
    assert not hook.live  # every buffer went back to the pool
    assert torch.cuda.memory_allocated() == before
