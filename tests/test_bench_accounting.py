"""The cost accounting behind bench.py's roofline and accuracy fields (CPU)."""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1704_08897_gb300 import synth  # noqa: E402


def test_algorithmic_cost_per_kernel_kind():
    probs = [synth.circle(64), synth.wobbly(128, 0)]
    nodes = 64 * 64 + 128 * 128
    # double-float CG vectors: 8 bytes per node per vector
    assert bench.algorithmic_cost(probs, "stencil") == (33 * nodes, "byte")
    assert bench.algorithmic_cost(probs, "update") == (48 * nodes, "byte")
    # 64 and 128 do not fold: all slicing is the unfolded kind
    assert bench.algorithmic_cost(probs, "split") == (16 * nodes, "byte")
    assert bench.algorithmic_cost(probs, "split", low=True) == (20 * nodes, "byte")
    assert bench.algorithmic_cost(probs, "fold") == (0, "byte")
    big = [synth.wobbly(256, 1)]
    assert bench.algorithmic_cost(big, "fold") == (16 * 256 * 256, "byte")
    assert bench.algorithmic_cost(probs, "unfold") == (25 * nodes, "byte")
    # stage s contracts one axis: 2 nx ny n_axis flop, x for stages 0 and 2, y for 1 and 3
    p = synth.wobbly(128, 0)
    assert bench.algorithmic_cost([p], "prec_stage0") == (2 * 128 ** 3, "flop")
    assert bench.algorithmic_cost([p], "prec_stage3") == (2 * 128 ** 3, "flop")
    assert bench.algorithmic_cost([p], "output") == (None, None)


def test_issued_tensor_flop_counts_ten_slice_products_on_padded_tiles():
    p = synth.wobbly(192, 1)  # padded to 256 on every axis
    assert bench.issued_tensor_flop([p], "prec_stage1", fold=False) == 2 * 10 * 256 ** 3
    # folded: four mirror classes of 96 x 96 nodes, each padded to 128 (half the products)
    assert bench.issued_tensor_flop([p], "prec_stage1", fold=True) == 4 * 2 * 10 * 128 ** 3
    q = synth.wobbly(128, 2)  # no padding; 64-node classes would pad back to 128: not folded
    assert bench.mirror_classes(128) == [128]
    assert bench.issued_tensor_flop([q], "prec_stage2") == 10 * bench.algorithmic_cost([q], "prec_stage2")[0]


def test_mirror_classes_follow_the_padding_rule():
    assert bench.mirror_classes(512) == [256, 256]
    assert bench.mirror_classes(255) == [128, 128]   # odd: the middle node is in the even class
    assert bench.mirror_classes(300) == [300]        # 150 pads to 256, twice 512 > 384
    assert bench.mirror_classes(512, fold=False) == [512]


def test_error_vs_oracle_is_the_max_norm_relative_error_over_unknowns():
    p = synth.circle(64)
    ref = np.linspace(-2.0, 3.0, 64 * 64).reshape(64, 64)
    known = np.zeros((64, 64), bool)
    from oracle import biharmonic as ob
    known[:] = ob.known_mask(p.phi.astype(np.float64), p.direction)
    ans = ref.copy()
    u = np.argwhere(~known)[0]
    ans[tuple(u)] += 3e-5                      # an error at one unknown node
    k = np.argwhere(known)[0]
    ans[tuple(k)] += 1.0                       # known nodes are not counted
    rep = bench.error_vs_oracle([p], [ans], [ref], "mixed_bf16")
    assert abs(rep["max_rel"] - 1e-5) < 1e-12  # 3e-5 / max |ref| (= 3)
    assert rep["bound"] == 1e-5 and rep["within"] and rep["problems"] == 1
    assert bench.error_vs_oracle([p], [ans], [ref], "fp32")["within"] is False
