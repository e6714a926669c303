"""What the trained network gains over the method without it: FastDSAC
trained on the GPU for a short wall-clock budget against the reactive
goal-seeking controller, on the same held-out maps, same episodes and the
same FP64 success reduction."""
import pytest

pytestmark = pytest.mark.gpu


def test_trained_policy_beats_reactive_controller():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_15846_b300 import train as TR
    cfg = TR.TrainConfig(time_budget_s=25.0, eval_every_s=1e9, n_eval=500)
    reactive, _ = TR.evaluate_reactive(cfg)
    res = TR.train(cfg, log=lambda *a: None)
    trained = res["history"][-1]["success"]
    print(f"held-out success: reactive {reactive:.3f}, trained (25 s) {trained:.3f}")
    assert trained > reactive + 0.1


def test_bf16_and_fp32_policy_paths_reach_equal_success():
    """The fused-rollout claim "at equal eval success": one trained policy
    (paper TurtleBot2 preset, 12 s of training) evaluated on the same 1000
    episodes through the BF16 tensor-core path and the plain FP32 path."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_15846_b300 import flashnav
    from paper_2606_15846_b300 import train as TR
    cfg = TR.paper_config("turtlebot2", time_budget_s=12.0, threshold=2.0, eval_every_s=1e9)
    res = TR.train(cfg, log=lambda *a: None, keep_policy=True)
    pol = res["policy"]
    s16, _ = TR.evaluate_policy(cfg, pol, fp32=False)
    s32, _ = TR.evaluate_policy(cfg, pol, fp32=True)
    flashnav.load().nav_policy_free(pol)
    print(f"success: BF16 tensor cores {s16:.3f}, FP32 {s32:.3f}")
    assert s16 > 0.6 and abs(s16 - s32) <= 0.03
