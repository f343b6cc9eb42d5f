"""The first-order manifold optimisation (Alg. 1) of the CUDA path against the oracle (needs a GB300).

Every iteration steps along -grad f with the energy-decrease line search; on a soft 3x3x3 lattice it converges in
about ten iterations and ten halvings each, which both paths must reproduce: the same iteration and halving counts,
positions to 1e-9 (FP64 path) and 1e-4 (mixed path) of the scene size. The direction involves no FP32 stage, so
the mixed path only differs in the line search's FP64 sums being the same as well.
"""
import numpy as np
import pytest

import oracle
import paper_2308_10459_gb300 as pkg
from paper_2308_10459_gb300 import build as bmod
from paper_2308_10459_gb300 import scenes

pytestmark = pytest.mark.gpu
TOL = {pkg.BDEM_FP64: 1e-9, pkg.BDEM_MIXED: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bmod.build()
    pkg.load()
    oracle.build()


@pytest.mark.parametrize("prec", [pkg.BDEM_FP64, pkg.BDEM_MIXED])
@pytest.mark.parametrize("graph", [True, False])
def test_first_order_matches_the_oracle(prec, graph):
    sc = scenes.cube_lattice(nx=3, E=1e5, z_bottom=0.006, k_ground=1e6, optimizer=1, newton_max_iter=300)
    o = oracle.OracleSim(sc)
    sim = pkg.Sim(sc, precision=prec)
    sim.set_step_graph(graph)
    L = float(np.linalg.norm(sc.pos.max(0) - sc.pos.min(0)))
    for k in range(4):
        so = o.step(1)[0][0]
        sg = sim.step(1)[0]
        assert sg["pcg_iters"] == 0
        assert (sg["newton_iters"], sg["ls_halvings"]) == (so["newton_iters"], so["ls_halvings"]), k
        st = sim.read_state()
        assert np.abs(st["pos"] - o.p).max() <= TOL[prec] * L, k
    sim.close()
