"""Host-side helpers of bench.py (no GPU): the comment-free source hash that
keys the committed ncu traffic figure."""
import bench


def test_strip_comments_keeps_code_and_literals():
    src = ('int a = 1; // note\n'
           '/* block\n   comment */ const char *s = "a // b /* c */";\n'
           "char q = '\"';  \n"
           '\n'
           '  int b; /* t */\n')
    assert bench.strip_comments(src) == ('int a = 1;\n'
                                         ' const char *s = "a // b /* c */";\n'
                                         "char q = '\"';\n"
                                         '  int b;')


def test_comment_edits_do_not_change_the_stripped_source():
    a = "x = f(y);  // Algorithm 1\nz = 2;\n"
    b = "// a new line of commentary\nx = f(y);  /* reworded */\n\nz = 2;\n"
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments("x = f(y);\nz = 3;\n") != bench.strip_comments(a)


def test_kernel_source_hash_is_stable():
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    assert len(bench.kernel_source_hash()) == 16
