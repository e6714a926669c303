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
