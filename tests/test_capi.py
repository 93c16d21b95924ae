"""Host-side checks of the C ABI: the library loads without a GPU, exports
every entry point include/finger.h declares, and its pure-host helpers follow
the paper's memory formula.  No compute call is made here."""
import ctypes
import os
import re

import paper_2206_11408_gb300 as fg

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "finger.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(finger_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("finger_index_load", "finger_build_tables", "finger_search"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(fg._build.build())
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(fg.SIGNATURES)


def test_table_bytes_is_r_plus_2_floats_per_edge():
    # Supplementary F: (r + 2) * |E| * sizeof(float)
    assert fg.table_bytes(1_000_000, 32, 64) == 66 * 32_000_000 * 4
    assert fg.table_bytes(10_000, 32, 16) == 18 * 320_000 * 4
    # reduced precision: 16-byte aligned FP8 codes + two FP32 scalars
    # LP: FP8 codes of 64 slots (deg0 > 32) x 32 codes per node in the tensor
    # cores' operand order, plus the FP32 scalars of every edge slot
    assert fg.table_bytes(1_200_000, 48, 32, lp=True) == 64 * 32 * 1_200_000 + 8 * 1_200_000 * 48
    assert fg.table_bytes(1_000_000, 32, 64, lp=True) == 32 * 64 * 1_000_000 + 8 * 1_000_000 * 32


def test_status_strings():
    L = fg.lib()
    for s in range(9):
        assert L.finger_status_str(s)


def test_argument_errors_are_reported_before_any_device_work():
    """Bad arguments of the index-free merge and of the visited-slot option
    come back as FINGER_ERR_INVALID_ARG (1) from host-side checks, so they are
    testable without a GPU."""
    L = fg.lib()
    one = (ctypes.c_int64 * 1)(0)
    neg = (ctypes.c_int64 * 2)(0, -5)
    p = ctypes.c_void_p(16)   # never dereferenced: the checks reject first
    args = dict(ids=p, d=p, S=1, nq=4, K=10, offs=one, oi=p, od=p)

    def merge(**kw):
        a = dict(args, **kw)
        return L.finger_merge_topk(a["ids"], a["d"], a["S"], a["nq"], a["K"], a["offs"],
                                   a["oi"], a["od"], None)

    assert merge(S=0) == 1 and merge(S=65) == 1
    assert merge(K=0) == 1 and merge(K=1025) == 1
    assert merge(nq=-1) == 1
    assert merge(offs=None) == 1
    assert merge(S=2, offs=neg) == 1
    assert merge(ids=None) == 1 and merge(od=None) == 1
    assert merge(nq=0) == 0                       # nothing to merge
    assert L.finger_set_visited_slots(None, 0) == 1
