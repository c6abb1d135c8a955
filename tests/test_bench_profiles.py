"""The link between the committed ncu summaries and the kernel sources (CPU).

bench.py reports a kernel's DRAM traffic from a committed capture only while
the kernels' code hashes to the values recorded with it; the hash is taken
over the code without comments, so that editing a comment keeps the capture.
"""
import os
import re

import bench


def test_code_of_drops_comments_and_keeps_literals():
    src = ('int a = 1;  // trailing\n/* block\n   comment */ const char *s = "x // y /* z */";\n'
           "char q = '/';\tint b = a /2;\n")
    assert bench.code_of(src) == ('int a = 1; const char *s = "x // y /* z */"; '
                                  "char q = '/'; int b = a /2;")


def test_comment_edits_keep_the_hash_and_code_edits_change_it():
    a = "__global__ void k(float *x) {\n    x[0] = 1.f;   // one\n}\n"
    b = "// the kernel\n__global__ void k(float *x) {\n    /* set */ x[0] = 1.f;\n}\n"
    c = "__global__ void k(float *x) {\n    x[0] = 2.f;\n}\n"
    assert bench.code_of(a) == bench.code_of(b) != bench.code_of(c)


def test_every_profile_names_each_kernel_source_once():
    names = {os.path.basename(p) for p in bench.KERNEL_SOURCES}
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")
    for f in sorted(os.listdir(root)):
        with open(os.path.join(root, f)) as fh:
            text = fh.read()
        hashes = {}
        for line in text.splitlines():
            bench.capture_hashes(line, hashes)
        assert set(hashes) == names, f
        assert all(re.fullmatch(r"[0-9a-f]{16}", v) for v in hashes.values()), f
