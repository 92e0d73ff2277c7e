"""Host-side logic of bench.py that needs no GPU: the kernel-code hash that keys the committed
DRAM-traffic figures to the code they were measured on."""

import os
import re

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
