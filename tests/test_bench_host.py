"""Host-side pieces of bench.py (no GPU): the recorded DRAM traffic is keyed
by a digest of the pair kernel's code, which comments and layout must not
change, and the record's capture commands follow the profiling rules."""
import json
import os

import bench


def test_kernel_digest_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    src = {}
    for rel in bench.PAIR_SOURCES:
        with open(os.path.join(bench.ROOT, rel), encoding="utf-8") as f:
            src[rel] = f.read()
    base = bench.pair_kernel_digest()

    def digest_of(texts):
        root = tmp_path / str(len(list(tmp_path.iterdir())))
        for rel, t in texts.items():
            p = root / rel
            p.parent.mkdir(parents=True, exist_ok=True)
            p.write_text(t, encoding="utf-8")
        monkeypatch.setattr(bench, "ROOT", str(root))
        return bench.pair_kernel_digest()

    commented = {rel: "// a note\n" + t.replace("\n", "  \n", 3) for rel, t in src.items()}
    assert digest_of(commented) == base
    changed = dict(src)
    rel0 = bench.PAIR_SOURCES[0]
    changed[rel0] = src[rel0].replace("constexpr int PAIR_T = 256;", "constexpr int PAIR_T = 128;")
    assert changed[rel0] != src[rel0]
    assert digest_of(changed) != base


def test_traffic_record_is_well_formed():
    with open(bench.TRAFFIC_FILE) as f:
        rec = json.load(f)
    for name in ("mapping_64x100000", "window_10x50000", "lidar_street_8x20000"):
        ent = rec[name]
        assert ent["bytes_per_launch"] == ent["read"] + ent["write"] > 0
        assert "--clock-control none" in ent["command"] and "-c 1" in ent["command"]
        assert len(ent["source_sha256"]) == 64


def test_both_roofline_bounds():
    import numpy as np
    assert bench.label_row_bytes(19, 1) == 48 and bench.label_row_bytes(19, 0) == 80
    assert bench.label_row_bytes(0, 0) == 0 and bench.label_row_bytes(4, 0) == 16
    flat = dict(n_points=np.array([100, 200, 300]), edges=np.array([[0, 1], [1, 2]]), sem_dim=19,
                P=dict(sem_bf16=1), color=False)
    b = bench.pair_bounds(flat, 1e6, 80.0)
    assert b["algorithmic_bytes_per_launch"] == (300 + 500) * (16 + 48)
    assert abs(b["fp32_pair_terms_per_s"] - 80e12 / bench.FLOPS_PER_PAIR) < 1.0
    assert b["hbm_pair_terms_per_s"] == 1e6 / (b["algorithmic_bytes_per_launch"] / (b["hbm_gbs"] * 1e9))
    assert b["lower"] in ("fp32", "hbm")
