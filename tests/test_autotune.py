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
    assert set(shapes) == {"rows_per_block", "images_per_block", "row_pairs_per_block", "solve_grid",
                           "solve_tensor_cores"}
    assert shapes["solve_tensor_cores"] == 0  # not chosen by the tuner (it rounds differently)
    D1, x1, _, _, _ = plan.run_pair(Rt, St)
    torch.cuda.synchronize()
    assert np.array_equal(D1.cpu().numpy(), D0)
    assert np.array_equal(x1.cpu().numpy(), x0)
    other = SfftPlan(n0, n1, 3, 3, 2, 1, 1)
    assert binding.sfft_plan_tuning(other.handle) == shapes
    other.close()
    plan.close()


@pytest.mark.parametrize("shape", [(4096, 4096), (512, 256), (64, 32)])
def test_every_launch_shape_gives_the_same_result(shape):
    """Each rows-per-block, images-per-block and row-pairs-per-block choice,
    set by hand, gives the built-in choice's results bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, binding
    n0, n1 = shape
    R = random_field(n0, n1, 31)
    S = 0.9 * np.roll(R, (1, 2), axis=(0, 1)) + 0.3 * random_field(n0, n1, 32)
    Rt, St = torch.from_numpy(R).float().cuda(), torch.from_numpy(S).float().cuda()
    mask = torch.from_numpy((np.random.default_rng(5).random((n0, n1)) > 0.05).astype(np.uint8)).cuda()
    plan = SfftPlan(n0, n1, 3, 3, 2, 1, 1)
    D0, x0, _, M0, _ = plan.run_pair(Rt, St, mask, keep_system=True)
    torch.cuda.synchronize()
    D0, x0, M0 = D0.cpu().numpy(), x0.cpu().numpy(), M0.cpu().numpy()
    for shapes in ([1, 1, 1, 0, 0], [2, 2, 2, 0, 0], [4, 3, 1, 0, 0], [16, 4, 4, 0, 0]):
        binding.sfft_plan_set_tuning(plan.handle, shapes)
        D1, x1, _, M1, _ = plan.run_pair(Rt, St, mask, keep_system=True)
        torch.cuda.synchronize()
        assert np.array_equal(M1.cpu().numpy(), M0), shapes
        assert np.array_equal(D1.cpu().numpy(), D0), shapes
        assert np.array_equal(x1.cpu().numpy(), x0), shapes
    plan.close()


def test_set_tuning_rejects_bad_shapes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, binding
    plan = SfftPlan(64, 64, 2, 2, 1, 1, 1)
    good = binding.sfft_plan_tuning(plan.handle)
    for bad in ({"rows_per_block": 3}, {"rows_per_block": 32}, {"rows_per_block": -1}, {"images_per_block": 5},
                {"row_pairs_per_block": -2}, {"solve_grid": 513}, {"solve_tensor_cores": 3}):
        with pytest.raises(binding.SfftError):
            binding.sfft_plan_set_tuning(plan.handle, bad)
        assert binding.sfft_plan_tuning(plan.handle) == good
    binding.sfft_plan_set_tuning(plan.handle, [2, 1, 1, 0, 0])
    assert binding.sfft_plan_tuning(plan.handle) == dict(zip(binding.TUNING_KEYS, [2, 1, 1, 0, 0]))
    plan.close()
