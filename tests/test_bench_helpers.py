"""Host logic of bench.py that needs no GPU: the digest that ties an ncu
traffic record to the kernel code it was taken on (comments and the
bounds-check build's branches ignored, code edits detected)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

BASE = """__global__ void k(int *a) {
    int i = threadIdx.x;
    a[i] = i;
}
"""


def _digest(tmp_path, text):
    p = tmp_path / "k.cu"
    p.write_text(text)
    return bench.source_digest(str(p))


def test_digest_ignores_comments_blank_lines_and_checked_branches(tmp_path):
    d0 = _digest(tmp_path, BASE)
    commented = "// header\n" + BASE.replace("int i = threadIdx.x;", "int i = threadIdx.x;   // the lane") + "\n\n"
    assert _digest(tmp_path, commented) == d0
    checked = BASE.replace("    a[i] = i;\n", "#if WV_CHECKED\n    if (i < 0) return;\n#endif\n    a[i] = i;\n")
    assert _digest(tmp_path, checked) == d0
    with_else = BASE.replace("    a[i] = i;\n", "#if WV_CHECKED\n    a[i] = -i;\n#else\n    a[i] = i;\n#endif\n")
    assert _digest(tmp_path, with_else) == d0


def test_digest_sees_code_edits(tmp_path):
    d0 = _digest(tmp_path, BASE)
    assert _digest(tmp_path, BASE.replace("a[i] = i;", "a[i] = 2 * i;")) != d0
    other_if = BASE.replace("    a[i] = i;\n", "#if WV_STRIP_H\n    a[i] = i;\n#endif\n")
    assert _digest(tmp_path, other_if) != d0   # only the WV_CHECKED switch is dropped
