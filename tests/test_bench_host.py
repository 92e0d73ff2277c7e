"""Host-side logic that needs no GPU: bench.py's kernel-code hash (it keys the committed
DRAM-traffic figures to the code they were measured on) and the binding's composite-key helpers."""

import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_strip_comments_keeps_code_and_literals():
    src = ('int a = 1; // note\n/* block\n comment */ const char* s = "x // y /* z */";\n'
           "char q = '\"'; char e = '\\''; int b;  // end")
    assert bench.strip_comments(src) == (
        'int a = 1; const char* s = "x // y /* z */"; char q = \'"\'; char e = \'\\\'\'; int b;')


def test_comment_and_whitespace_edits_do_not_change_the_code_text():
    a = "template <int N>\n__global__ void k(int* p) {  // one\n  p[0] = N;\n}\n"
    b = "// header\ntemplate <int N>\n__global__ void k(int* p) { /* two */\n    p[0] = N;   \n}"
    c = "template <int N>\n__global__ void k(int* p) {\n  p[0] = N + 1;\n}\n"
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments(a) != bench.strip_comments(c)


def test_traffic_lines_are_well_formed():
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return
    h = bench.kernel_source_hash()
    assert re.fullmatch(r"[0-9a-f]{16}", h)
    for line in open(p):
        if line.startswith("#") or not line.strip():
            continue
        m = re.fullmatch(r"kernel=(\S+) workload=(\S+) bytes_per_launch=(\d+) src=([0-9a-f]{16})\s*", line)
        assert m, line
        assert int(m.group(3)) > 0


def test_composite_view_and_key_width_checks_on_host():
    import torch

    import paper_2106_05123_gb300 as pdq
    f = torch.tensor([[3, 1], [1, 9]], dtype=torch.int32)
    k = pdq.composite_keys(f)
    assert k.dtype == torch.int64 and k.shape == (2,)
    assert k.view(torch.int32).view(2, 2).tolist() == [[3, 1], [1, 9]]
    for bad in (torch.zeros(4, dtype=torch.int32), torch.zeros((3, 3), dtype=torch.int32),
                torch.zeros((3, 2), dtype=torch.int64)):
        with pytest.raises(pdq.PdqError):
            pdq.composite_keys(bad)
    # a key-type override must match the element width
    assert pdq._key_code(torch.zeros(2, dtype=torch.int64), pdq.PDQ_I32I32) == pdq.PDQ_I32I32
    assert pdq._key_code(torch.zeros(2, dtype=torch.int32), pdq.PDQ_U32) == pdq.PDQ_U32
    with pytest.raises(pdq.PdqError):
        pdq._key_code(torch.zeros(2, dtype=torch.int32), pdq.PDQ_F32U32)
