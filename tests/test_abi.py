"""Host-side checks of the C ABI (no GPU): the library loads, exports every function declared
in include/blm.h, validates problems before touching a device, and its storage helpers give the
paper's worked example."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1702_01481_gb300", "libblm.so")

pytestmark = pytest.mark.skipif(not os.path.exists(LIB), reason="libblm.so not built")


def declared_functions():
    src = open(os.path.join(ROOT, "include", "blm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(blm_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    import ctypes
    lib = ctypes.CDLL(LIB)
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    import paper_1702_01481_gb300 as blm
    assert set(names) <= set(blm.EXPORTED)


def test_storage_figures_match_the_paper():
    import paper_1702_01481_gb300 as blm
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "memory_example.txt"))
            if l.strip() and not l.startswith("#")]
    for method, n, nb, no, gb in rows:
        digits = len(gb.split(".")[1])
        if method == "LM":
            got = blm.blm_lm_matrix_bytes(int(n)) / 1e9
        else:
            got = blm.blm_matrix_bytes_dominant(int(n), int(nb), int(no)) / 1e9
        assert round(got, digits) == float(gb)


@pytest.mark.parametrize("offs,nk,status", [
    ([0, 5, 5, 10], 2, 1),       # empty block
    ([0, 5, 11], 2, 1),          # does not end at n
    ([1, 5, 10], 2, 1),          # does not start at 0
    ([0, 5, 10], 0, 1),          # n_keep 0
])
def test_invalid_problems_are_rejected_on_the_host(offs, nk, status):
    import paper_1702_01481_gb300 as blm
    p = blm.make_problem(10, offs, nk)
    with pytest.raises(blm.BLMError) as e:
        blm.blm_create(p)
    assert e.value.status == status
    assert blm.blm_memory_estimate(p) == 0


def test_unsupported_combinations():
    import paper_1702_01481_gb300 as blm
    p = blm.make_problem(10, [0, 5, 10], 2, precision=blm.BLM_PREC_BF16X4, input_type=blm.BLM_IN_F64)
    with pytest.raises(blm.BLMError) as e:
        blm.blm_create(p)
    assert e.value.status == blm.BLM_ERR_UNSUPPORTED


def test_memory_estimate_grows_with_the_problem():
    import paper_1702_01481_gb300 as blm
    a = blm.blm_memory_estimate(blm.make_problem(2048, [128 * i for i in range(17)], 10))
    b = blm.blm_memory_estimate(blm.make_problem(4096, [256 * i for i in range(17)], 10))
    assert 0 < a < b
