"""The benchmark's algorithmic flop table equals the oracle's counts, and its
per-voxel bookkeeping follows the status-word layout of include/gsm.h."""
import numpy as np

import oracle as O
import synth


def test_bench_flop_table_equals_the_oracle_counts():
    import bench
    prm = (70.0, 0.3, 0.1, 1.0, 5.0)
    eps, zn = synth.material_batch(4, seed=2)
    s, z = O.update(O.KIND_NORTON, prm, eps, zn, 0.01)
    c = O.flop_pieces(prm, eps[0], zn[0], z[0][[0, 1, 3, 4, 5]], 0.01)
    for piece, k in c.items():
        assert bench.ALG_FLOPS[piece] == k["add"] + k["mul"] + k["div"] + k["sqrt"], piece
        assert bench.ALG_POWS[piece] == k["pow"], piece


def test_alg_flops_from_status_words():
    """Status word: bits 0-7 line-search steps, 8-15 Newton steps (FP64
    corrections included), 20-23 FP64 corrections."""
    import bench
    A = bench.ALG_FLOPS
    st = np.array([3 | (2 << 8), 5 | (1 << 8)], dtype=np.int32)
    f64, f32, p64, p32 = bench.alg_flops_per_voxel(st, "fp64")
    expect = np.mean([A["predictor"] + 3 * A["line"] + 2 * A["newton"] + A["stress"],
                      A["predictor"] + 5 * A["line"] + 1 * A["newton"] + A["stress"]])
    assert f64 == expect and f32 == 0.0 and p64 == np.mean([3 * 3 + 2 * 3, 5 * 3 + 3])
    st = np.array([4 | (3 << 8) | (1 << 20)], dtype=np.int32)  # 2 FP32 Newton steps + 1 correction
    f64, f32, p64, p32 = bench.alg_flops_per_voxel(st, "fp32fix")
    assert f64 == A["residual"] + 5 + A["stress"] and p64 == 1
    assert f32 == A["predictor"] + 4 * A["line"] + 2 * A["newton"] + A["subst"]


def test_alg_flops_count_the_segment_model():
    """Bits 24-30: scalar iterations of the segment model (FP32 flops and
    exponentials); the FP64 mode adds one FP64 refinement step."""
    import bench
    A = bench.ALG_FLOPS
    st = np.array([2 | (1 << 8) | (4 << 24)], dtype=np.int32)
    f64, f32, p64, p32 = bench.alg_flops_per_voxel(st, "fp64")
    assert f64 == A["predictor"] + 2 * A["line"] + A["newton"] + A["stress"] + bench.MODEL64_FLOPS
    assert f32 == 4 * bench.MODEL_FLOPS and p32 == 4 * bench.MODEL_POWS
    st = np.array([2 | (2 << 8) | (1 << 20) | (4 << 24)], dtype=np.int32)
    f64, f32, p64, p32 = bench.alg_flops_per_voxel(st, "fp32fix")
    assert f32 == A["predictor"] + 2 * A["line"] + A["newton"] + A["subst"] + 4 * bench.MODEL_FLOPS
