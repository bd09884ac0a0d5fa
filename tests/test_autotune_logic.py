"""Host logic of the batched form's autotuner (no GPU): which knob values a trial may take
for a given precision and batch, and the default choices. The timing itself runs in
tests/test_gpu_batched.py."""
import torch

from paper_1310_7202_gb300 import autotune


def _probs(shapes):
    return [{"A": torch.empty(m, n), "k": k, "l": l, "seed": i}
            for i, (m, n, k, l) in enumerate(shapes)]


def test_every_knob_has_its_default_among_its_values():
    for knob, values in autotune.KNOBS.items():
        assert autotune.DEFAULTS[knob] in values


def test_tensor_core_and_simt_knobs_follow_the_precision():
    p = _probs([(300, 200, 20, 30)])
    # mixed: the Y and C products run on the tensor cores, their SIMT tiles are fixed
    assert not autotune._applicable("gemm_tile_y", "mixed", p, 1)
    assert not autotune._applicable("gemm_tile_c", "mixed", p, 1)
    assert autotune._applicable("umma_ctas_y", "mixed", p, 2)
    assert autotune._applicable("umma_ctas_c", "mixed", p, 2)
    # plain FP32: no tensor-core ring to size
    assert autotune._applicable("gemm_tile_y", "f32", p, 1)
    assert not autotune._applicable("umma_ctas_y", "f32", p, 2)
    assert not autotune._applicable("umma_ctas_c", "f32", p, 2)


def test_l_product_tile_only_matters_above_k_64():
    assert not autotune._applicable("gemm_tile_l", "f32", _probs([(300, 200, 64, 74)]), 1)
    assert autotune._applicable("gemm_tile_l", "f32", _probs([(300, 200, 66, 76)]), 1)


def test_lu_rows_per_cta_respects_the_cluster_limit():
    # 16 CTAs per cluster: 256-row CTAs reach 4096 rows, 512-row CTAs 8192
    assert autotune._applicable("lu_rows_per_cta", "f32", _probs([(4096, 1000, 20, 30)]), 256)
    assert not autotune._applicable("lu_rows_per_cta", "f32", _probs([(5000, 1000, 20, 30)]), 256)
    assert autotune._applicable("lu_rows_per_cta", "f32", _probs([(5000, 1000, 20, 30)]), 512)
