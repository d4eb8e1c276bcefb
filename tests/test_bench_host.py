"""Host-side pieces of bench.py that its reported numbers depend on (no GPU).

* code_tokens / kernel_sources_sha1: the ncu traffic record is reported only
  while the kernel code equals the captured code; comments may change, code
  may not.
* kernel_rooflines: the algorithmic multiply counts per kernel kind for both
  layer-3 forms, checked against the per-row formulas written out here.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def test_code_tokens_drop_comments_but_not_strings():
    a = 'int x = 1; // note\n/* block\n */ const char *s = "a // b /* c */";\n'
    b = 'int x = 1;\nconst char *s = "a // b /* c */";'
    assert bench.code_tokens(a) == bench.code_tokens(b)
    assert "// b /* c */" in bench.code_tokens(a)
    assert bench.code_tokens("int x = 1;") != bench.code_tokens("int x = 2;")
    assert bench.code_tokens("char q = '\"'; int y;") == "char q = '\"'; int y;"


def test_kernel_fingerprint_matches_the_committed_traffic_record_format():
    fp = bench.kernel_sources_sha1()
    assert len(fp) == 40 and int(fp, 16) >= 0


INFO = {"producer_window_rows": 11444, "state_compute_rows": 1322, "deep_compute_rows": 156,
        "deep_tail_rows": 1433, "state_rows": 107075, "deep_head_runs": 1305}


@pytest.mark.parametrize("k,min_k", [(8, 9), (10, 9), (10, 21), (12, 6)])
def test_mid_layer_multiply_counts_per_layer3_form(k, min_k):
    info = dict(INFO, pair_layer3_min_k=min_k, head_table=0, deep_heads=1300)
    c, D, DC, H = 256, 1322, 156, 1305
    kt = {"mid_layer": (1.0, k - 5 - (1 if min_k <= k else 0)), "third_layer": (1.0, 1)}
    out = bench.kernel_rooflines(info, k, c, 2, 100000, kt, 1, 6000.0, 1e11)
    mid = DC * (c + k)
    if min_k <= k:
        # layer 4 reads pair windows (3 products a point), then plain middle layers
        launches = [DC * (3 * c + k)] + [mid] * (k - 7)
        assert out["third_layer"]["alg_gf_mults_per_launch"] == D * (k + k * k)
    else:
        # layer 3 per point (2 a point and row, 1 a point and head run), then plain
        launches = [D * (k + 2 * c) + H * c] + [mid] * (k - 6)
        assert "third_layer" not in out
    assert out["mid_layer"]["alg_gf_mults_per_launch"] == int(sum(launches) / len(launches))
