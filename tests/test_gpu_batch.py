"""The batched persistent launch: thousands of uneven systems, each solved by the whole method in one
CTA, against the oracle (backward error per system, agreement with GEPP), plus autotuning and graph replay."""
import numpy as np
import pytest
import torch

from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W
from paper_1406_5802_gb300.batch import CONFIGS, BatchedSolver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1406_5802_gb300 import build as B
    B.build()
    rmge.load_library()


def _batch(count, lo, hi, seed):
    sizes = W.batch_sizes(count, lo, hi, seed)
    systems = W.batch_systems(sizes, seed + 1)
    return [a for a, _, _ in systems], [b for _, b, _ in systems]


@pytest.mark.parametrize("config", sorted(CONFIGS))
def test_batched_matches_oracle(orc, config):
    As, bs = _batch(60, 1, 300, seed=41)  # includes n = 1 and ragged sizes around the 32-column blocks
    bs_ = BatchedSolver(As, bs, seed=9, max_sweeps=40, be_tol=1e-13)
    bs_.launch(config, 2 * 152)
    torch.cuda.synchronize()
    info = bs_.info.cpu().numpy()
    berr = bs_.berr.cpu().numpy()
    assert np.all(info == 0)
    for i, (a, b) in enumerate(zip(As, bs)):
        x = bs_.solution(i).cpu().numpy().reshape(-1, 1)
        be = orc.backward_error(a, x, b)
        assert be <= 1e-13, (i, a.shape[0], be, berr[i])
        assert berr[i] <= 1e-13
        assert abs(berr[i] - be) <= 0.5 * be + 1e-17


def test_batched_graph_replay_and_tuning(orc):
    As, bs = _batch(400, 32, 160, seed=7)
    s = BatchedSolver(As, bs, seed=3, max_sweeps=40)
    entry = s.tune(reps=1, use_cache=False)
    assert entry["config"] in CONFIGS
    s.capture()
    for _ in range(2):  # the queue re-arms itself: replays repeat the same work
        s.x.zero_()
        s.run()
        torch.cuda.synchronize()
        assert np.all(s.info.cpu().numpy() == 0)
        assert np.all(s.berr.cpu().numpy() <= 1e-13)
    for i in (0, 57, 399):
        x = s.solution(i).cpu().numpy().reshape(-1, 1)
        assert orc.backward_error(As[i], x, bs[i]) <= 1e-13


def test_uneven_batch_all_systems_reach_target(orc):
    """The uneven-batch workload (n ~ U{32..512}, A[0,0] scaled by 1e-10): every system reaches the FP64 target,
    through FP32 factors with FP64 sweeps, a fresh multiplier, or the FP64 fallback."""
    As, bs = _batch(120, 32, 512, seed=W.SEED_BASE + 4)
    s = BatchedSolver(As, bs, seed=W.SEED_BASE + 4, max_sweeps=40)
    s.launch(1, 2 * 152)
    torch.cuda.synchronize()
    assert np.all(s.info.cpu().numpy() == 0)
    berr = s.berr.cpu().numpy()
    assert np.all(berr <= 1e-13), (np.argmax(berr), float(np.max(berr)))
    for i in range(0, 120, 7):
        x = s.solution(i).cpu().numpy().reshape(-1, 1)
        assert orc.backward_error(As[i], x, bs[i]) <= 1e-13


def test_fp64_fallback_shares_its_product(orc):
    """Systems with kappa(A) = 1e12 defeat every FP32 draw (kappa u_32 >> 1) and end in the FP64 fallback.
    The first of them in a launch posts its FP64 product A G as row blocks that the other CTAs take
    between systems; the second finds the launch's job slot taken and computes its product alone.  Both
    reach the FP64 target, and a second launch (the slot re-armed) repeats them."""
    As, bs = [], []
    for i, n in enumerate([300, 257, 40, 100, 64, 129, 200, 33]):
        if i < 2:
            A, B = W.orthogonal_factor_system(n, 1, 1e-12, seed=71 + i)
        else:
            A, B = W.gaussian_system(n, 1, seed=80 + i)
        As.append(A)
        bs.append(B)
    for config in sorted(CONFIGS):
        s = BatchedSolver(As, bs, seed=5, max_sweeps=40, be_tol=1e-13)
        for _ in range(2):
            s.x.zero_()
            s.launch(config, 2 * 152)
            torch.cuda.synchronize()
            info = s.info.cpu().numpy()
            berr = s.berr.cpu().numpy()
            assert np.all(info == 0), (config, info)
            assert np.all(berr <= 1e-13), (config, berr)
            for i in range(len(As)):
                x = s.solution(i).cpu().numpy().reshape(-1, 1)
                assert orc.backward_error(As[i], x, bs[i]) <= 1e-13, (config, i)
