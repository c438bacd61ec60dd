"""Host-side logic that needs no GPU: the autotuner's search space and its
restriction, the benchmark's kernel naming and tree options, and the
combination of sharded fused-MSE adjoints."""
import pytest
import torch

import bench
from paper_2208_10295_gb300 import tune
from paper_2208_10295_gb300.torch_api import combine_mse


def test_candidates_cover_the_space_and_respect_restrictions():
    full = list(tune.candidates(points=True))
    assert full and all(256 <= c["block_threads"] * c["blocks_per_sm"] <= 2048 for c in full)
    # the cost schedules need the Morton-ordered base order
    assert all(c["ray_order"] == 1 for c in full if c["schedule"] != "morton")
    # without a point cloud the fused and separate scatter are the same cast
    assert all(c["fused_scatter"] == 1 for c in tune.candidates(points=False))
    assert not any(c["traversal"] == 3 for c in tune.candidates(points=True, wide8=False))
    only = list(tune.candidates(points=True, restrict=bench.HEADLINE_LAUNCH))
    assert only and all(c["traversal"] == 2 and c["block_threads"] == 256 and c["blocks_per_sm"] == 2
                        for c in only)
    assert {(c["ray_order"], c["schedule"], c["fused_scatter"]) for c in only} == \
        {(c["ray_order"], c["schedule"], c["fused_scatter"]) for c in full
         if c["traversal"] == 2 and c["block_threads"] == 256 and c["blocks_per_sm"] == 2}


def test_kernel_name_follows_the_register_variant():
    assert bench.kernel_name({"block_threads": 256, "blocks_per_sm": 2, "traversal": 2}) == "k_cast<0, 2, 2>"
    assert bench.kernel_name({"block_threads": 128, "blocks_per_sm": 4, "traversal": 2}) == "k_cast<0, 2, 2>"
    assert bench.kernel_name({"block_threads": 256, "blocks_per_sm": 3, "traversal": 3}) == "k_cast<0, 3, 3>"
    assert bench.kernel_name({"block_threads": 256, "blocks_per_sm": 8, "traversal": 2}) == "k_cast<0, 4, 2>"


def test_capture_constants_name_the_benchmark_trees():
    assert bench.NCU_TRAFFIC["tree"] == bench.CFG1_TREE
    assert bench.NCU_FP32["tree"] == bench.CFG1_TREE
    assert bench.NCU_CITY_UNITS["tree"] == bench.CITY_TREE
    assert "treelet rounds" in bench.tree_name(bench.CITY_TREE)


def test_combine_mse_weights_parts_by_their_counts():
    parts = [(torch.tensor([2.0]), torch.tensor([[1.0, 0.0]]), torch.tensor([4.0]), torch.tensor([1])),
             (torch.tensor([5.0]), torch.tensor([[0.0, 3.0]]), torch.tensor([1.0]), torch.tensor([3])),
             (torch.tensor([9.0]), torch.tensor([[7.0, 7.0]]), torch.tensor([9.0]), torch.tensor([0]))]
    loss, gT, gg = torch.zeros(1), torch.zeros(1, 2), torch.zeros(1)
    n = combine_mse(parts, loss, gT, gg)
    assert float(n) == 4.0
    assert loss.item() == pytest.approx((2.0 * 1 + 5.0 * 3) / 4)
    assert gT.flatten().tolist() == pytest.approx([0.25, 2.25])
    assert gg.item() == pytest.approx((4.0 + 3.0) / 4)
    # no beams anywhere: zeros, not NaN
    n0 = combine_mse([(torch.tensor([1.0]), torch.ones(1, 2), torch.ones(1), torch.tensor([0]))], loss, gT, gg)
    assert float(n0) == 0.0 and loss.item() == 0.0 and not gT.any() and gg.item() == 0.0
