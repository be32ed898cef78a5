"""The algorithmic counts behind bench.py's rooflines, against hand counts of the frame
workload's sizes: 1312 B and 55,936 flops per live sample."""
import os
import sys

from paper_2306_16541_gb300 import synth

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_frame_workload_counts():
    s = synth.config_frame512()["subject"]
    # 24 bones x 8 corners x 4 B + 16 levels x 8 corners x 2 features x 2 B + 16 B in + 16 B out
    assert bench.field_bytes_per_sample(s, table_bytes=2) == 768 + 512 + 32 == 1312
    # residual: 39 -> 64, 64 -> 64, 64 -> 64, (64 + 39) -> 64, 64 -> 3; canonical: 32 -> 64,
    # 64 -> 64 twice, 64 -> 4; two flops per multiply-add
    res = 39 * 64 + 64 * 64 + 64 * 64 + 103 * 64 + 64 * 3
    can = 32 * 64 + 2 * 64 * 64 + 64 * 4
    assert bench.mlp_flops_per_sample(s) == 2 * (res + can) == 55936


def test_counts_follow_the_subject():
    s = dict(synth.config_frame512()["subject"])
    s["hash_levels"] = 8
    assert bench.field_bytes_per_sample(s, table_bytes=4) == 768 + 8 * 8 * 2 * 4 + 32
    s["res_enabled"] = 0
    assert bench.mlp_flops_per_sample(s) == 2 * (16 * 64 + 2 * 64 * 64 + 64 * 4)


def test_counts_follow_the_feature_count():
    # four features per level: the first canonical layer sees L x 4 inputs, each corner read is 4 x 2 B
    s = dict(synth.config_frame512()["subject"])
    s["hash_feats"] = 4
    assert bench.field_bytes_per_sample(s, table_bytes=2) == 768 + 16 * 8 * 4 * 2 + 32
    res = 39 * 64 + 64 * 64 + 64 * 64 + 103 * 64 + 64 * 3
    can = 64 * 64 + 2 * 64 * 64 + 64 * 4
    assert bench.mlp_flops_per_sample(s) == 2 * (res + can)
