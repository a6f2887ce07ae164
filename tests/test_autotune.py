"""sfft_plan_autotune: launch shapes chosen by timing, results unchanged.

The tuned shapes only change how the work is split into blocks (rows per
block, images per block, row pairs per block, solve grid), so a tuned plan
must give bit-identical results, and a later plan of the same size, types
and D_K must start with the shapes found."""
import numpy as np
import pytest

from synth import random_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(256, 256), (96, 80)])
def test_autotune_keeps_results_and_is_remembered(shape):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, binding
    n0, n1 = shape
    R = random_field(n0, n1, 21)
    S = 0.9 * np.roll(R, (1, 2), axis=(0, 1)) + 0.3 * random_field(n0, n1, 22)
    Rt, St = torch.from_numpy(R).float().cuda(), torch.from_numpy(S).float().cuda()
    plan = SfftPlan(n0, n1, 3, 3, 2, 1, 1)
    D0, x0, _, _, _ = plan.run_pair(Rt, St)
    torch.cuda.synchronize()
    D0, x0 = D0.cpu().numpy(), x0.cpu().numpy()
    shapes = plan.autotune(Rt, St)
    assert set(shapes) == {"rows_per_block", "images_per_block", "row_pairs_per_block", "solve_grid"}
    D1, x1, _, _, _ = plan.run_pair(Rt, St)
    torch.cuda.synchronize()
    assert np.array_equal(D1.cpu().numpy(), D0)
    assert np.array_equal(x1.cpu().numpy(), x0)
    other = SfftPlan(n0, n1, 3, 3, 2, 1, 1)
    assert binding.sfft_plan_tuning(other.handle) == shapes
    other.close()
    plan.close()
