"""Host-side checks of tpa_cpi_step_noalloc that need no GPU: the n + m limit
its fixed 16 MiB scratch sets, and the refusal of in-place steps.

The library checks sizes and aliasing before any CUDA call, so these run on a
machine without a GPU through the C ABI.
"""
import ctypes

import pytest

C = 0.15


def lib():
    import paper_1708_02574_gb300 as tpa
    return tpa.library()


def call(n, m, x=None, y=None, r=None):
    L = lib()
    st = L.tpa_cpi_step_noalloc(ctypes.c_int64(n), ctypes.c_int64(m), None, None, None, ctypes.c_double(C),
                                x, y, r, None, None)
    return st, L.tpa_last_error().decode()


def fits(nm: int) -> bool:
    """True when n + m = nm passes the scratch-size check (the call then stops
    at the NULL arrays, before any CUDA work)."""
    n = min(nm, (1 << 31) - 1)
    st, msg = call(n, nm - n)
    assert st == 1, (st, msg)
    return "scratch" not in msg


def test_limit_is_about_134_million():
    lo, hi = 1, 1 << 31
    assert fits(lo) and not fits(hi)
    while hi - lo > 1:                      # the largest n + m accepted
        mid = (lo + hi) // 2
        if fits(mid):
            lo = mid
        else:
            hi = mid
    assert 133_500_000 < lo < 134_500_000, lo   # the figure include/tpa.h states
    assert fits(lo) and not fits(lo + 1)


@pytest.mark.parametrize("alias", ["x=y", "x=r", "y=r"])
def test_in_place_steps_are_refused(alias):
    a = ctypes.c_void_p(0x10000)
    b = ctypes.c_void_p(0x20000)
    c = ctypes.c_void_p(0x30000)
    x, y, r = {"x=y": (a, a, c), "x=r": (a, b, a), "y=r": (a, b, b)}[alias]
    st, msg = call(1024, 4096, x, y, r)
    assert st == 1 and "distinct" in msg, msg
