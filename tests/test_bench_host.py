"""Host-side logic of bench.py that needs no GPU."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_source_hash_ignores_comments_and_layout():
    import bench
    code = 'int f(int x) {\n  return x + 1;  // add one\n}\nconst char* s = "a // b /* c */";\n'
    edited = '/* header */\nint f(int x) {\n    return x + 1;  /* one */\n}\n' \
             'const char* s = "a // b /* c */";  // same string\n'
    assert bench._strip_comments(code) == bench._strip_comments(edited)
    assert '"a // b /* c */"' in bench._strip_comments(code)
    assert bench._strip_comments("x = '\\'' ; // q\ny") == "x = '\\'' ; y"
    assert bench._strip_comments("a = 1;") != bench._strip_comments("a = 2;")


def test_source_hash_is_stable():
    import bench
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()


def test_source_hash_over_named_files():
    import bench
    one = bench.kernel_source_hash(["resample3d.cu"])
    assert one == bench.kernel_source_hash(["resample3d.cu"])
    assert one != bench.kernel_source_hash(["resample3d.cu", "nfft_plan.cu"])
    assert one != bench.kernel_source_hash()
