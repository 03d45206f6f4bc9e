"""The C ABI library loads and exports every entry point include/*.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = "".join(open(os.path.join(ROOT, "include", f)).read() for f in sorted(os.listdir(os.path.join(ROOT, "include")))
                   if f.endswith(".h"))
    return sorted(set(re.findall(r"QUMOND_API\s+[\w\s\*]+?\b(qumond_\w+)\s*\(", text)))


def test_header_declares_the_six_path_calls():
    syms = declared_symbols()
    for name in ("qumond_deposit", "qumond_solve_newton", "qumond_source", "qumond_solve_mond", "qumond_forces",
                 "qumond_rotation_curve"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    lib_path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    import paper_1201_3185_gb300 as q
    assert sorted(q.EXPORTED) == declared_symbols()


def test_params_struct_matches_defaults():
    import paper_1201_3185_gb300 as q
    p = q.default_params()
    assert (p.n, p.ncycle, p.npre, p.npost) == (256, 6, 2, 2)
    assert p.G == pytest.approx(4.30e-3) and p.a0 == pytest.approx(3.6)
    assert p.deposit_shift == 24 and p.rc_box_frac == pytest.approx(0.2)


def test_guess_parameter_count():
    import paper_1201_3185_gb300 as q
    layers = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (192, 64), (64, 64),
              (96, 32), (32, 32), (48, 16), (16, 16)]
    assert q.Guess.num_params() == sum(27 * a * b + b for a, b in layers) + 17 == 1466065
