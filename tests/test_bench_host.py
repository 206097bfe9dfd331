"""Host-side helpers of bench.py (no GPU): the source hash that keeps stored
ncu counters tied to the code they were taken on."""
import bench


def test_code_text_drops_comments_keeps_literals():
    src = ('int a = 1; // note\n/* block\n   comment */ const char* s = "x // y /* z */";\n'
           'asm volatile("mov.u32 %0, 1; // ptx text" : "=r"(a));\nchar q = \'"\';\n\n')
    code = bench._code_text(src)
    assert "note" not in code and "block" not in code
    assert '"x // y /* z */"' in code and "// ptx text" in code
    assert "char q = '\"';" in code


def test_comment_edit_keeps_hash_code_edit_changes_it():
    base = "int f(int x) {\n  return x + 1;  // add one\n}\n"
    comment_only = "/* header */\nint f(int x) {\n  return x + 1;  // add 1\n}\n\n"
    one_token = "int f(int x) {\n  return x + 2;  // add one\n}\n"
    in_string = 'const char* p = "a // b";\n'
    in_string2 = 'const char* p = "a // c";\n'
    assert bench._code_text(base) == bench._code_text(comment_only)
    assert bench._code_text(base) != bench._code_text(one_token)
    assert bench._code_text(in_string) != bench._code_text(in_string2)


def test_oracle_timing_pieces_are_one_full_solve():
    """The reference arm times one oracle solve cut into pieces: for any piece
    count the pieces reproduce oracle.bie.solve exactly."""
    import numpy as np
    import workloads as W
    from oracle import bie as O
    g, f, ph = W.one_ellipse_640()
    om, U, psi = O.solve(g, f, ph)
    for k in (1, 2, 5):
        per, o, phases = bench.time_oracle_solve(g, f, ph, k)
        assert len(per) == k
        assert np.array_equal(o.omega, om) and np.array_equal(o.U, U) and np.array_equal(o.psi, psi)
