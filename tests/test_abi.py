"""C-ABI checks that need no GPU: the library loads, exports every function
include/amr_transfer.h declares, and rejects bad descriptors on the host
before any CUDA call (no side effects, *out stays NULL)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2504_15814_gb300 import binding as B
from paper_2504_15814_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(amr_[a-z_0-9]+)\s*\(", text, re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        pytest.skip("library not built")
    return B.lib()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    # the binding declares exactly what the header declares
    assert set(B.ENTRY_POINTS) <= set(names)


def test_status_strings(lib):
    for code, text in B.STATUS.items():
        assert lib.amr_status_string(code).decode() == text
    assert lib.amr_status_string(99).decode() == "unknown status"


def _create(items, U=4, cl=None, fl=None, abi=B.ABI_VERSION, precision=0, flags=0):
    arr, n = B._items_array(items)
    if cl is None:
        _, cl, fl = wl.make_items([it["face"] for it in items], [it["subface"] for it in items],
                                  [it["patch_size"] for it in items], [it["overlap"] for it in items],
                                  [it["order"] for it in items], U)
    desc = B.Desc(abi, U, precision, flags, n, ctypes.cast(arr, ctypes.c_void_p), cl, fl)
    h = ctypes.c_void_p(12345)
    st = B.lib().amr_transfer_plan_create(ctypes.byref(desc), ctypes.byref(h))
    return st, h


def _item(**kw):
    it = dict(face=0, subface=-1, patch_size=9, overlap=3, order=3, scheme=0, coarse_offset=0, fine_offset=0)
    it.update(kw)
    return it


@pytest.mark.parametrize("bad,status", [
    (dict(face=6), 1), (dict(face=-1), 1), (dict(subface=9), 1), (dict(subface=-2), 1),
    (dict(order=0), 1), (dict(order=4), 1), (dict(patch_size=0), 1), (dict(overlap=0), 1),
    (dict(patch_size=3), 2), (dict(overlap=6, patch_size=12), 2), (dict(overlap=4, patch_size=10), 2),
    (dict(overlap=5, patch_size=12, scheme=1), 2), (dict(patch_size=51), 2),
    (dict(order=2, overlap=1), 2), (dict(order=3, overlap=1), 2), (dict(scheme=2), 1), (dict(scheme=-1), 1),
    (dict(scheme=1, order=1), 2),
    (dict(coarse_offset=-1), 1), (dict(fine_offset=1), 1), (dict(coarse_offset=1), 1),
])
def test_invalid_items_rejected_on_host(lib, bad, status):
    st, h = _create([_item(**bad)] if "coarse_offset" not in bad and "fine_offset" not in bad else [_item(**bad)],
                    cl=2 * 3 * 81 * 4 if ("coarse_offset" in bad or "fine_offset" in bad) else None,
                    fl=9 * 2 * 3 * 81 * 4 if ("coarse_offset" in bad or "fine_offset" in bad) else None)
    assert st == status
    assert h.value is None


def test_bad_descriptor(lib):
    st, h = _create([_item()], abi=99)
    assert st == 1 and h.value is None
    st, h = _create([_item()], precision=7)
    assert st == 1
    st, h = _create([_item()], flags=2)
    assert st == 1
    assert lib.amr_transfer_plan_create(None, None) == 1
    assert lib.amr_transfer_plan_destroy(None) == 0
    assert lib.amr_transfer_plan_interpolate(None, None, None, None) == 1
    assert lib.amr_transfer_plan_restrict(None, None, None, None) == 1
    assert lib.amr_transfer_plan_get_info(None, None) == 1


def test_overlapping_outputs_rejected(lib):
    U = 2
    arr = 2 * 3 * 81 * U
    # two items writing the same fine face arrays
    items = [_item(subface=0, coarse_offset=0, fine_offset=0), _item(subface=1, coarse_offset=0, fine_offset=arr // 2)]
    st, _ = _create(items, U=U, cl=arr, fl=2 * arr)
    assert st == 1
    # two items restricting the same subface of one coarse face array
    items = [_item(subface=4, coarse_offset=0, fine_offset=0), _item(subface=4, coarse_offset=0, fine_offset=arr)]
    st, _ = _create(items, U=U, cl=arr, fl=2 * arr)
    assert st == 1
    # a whole-face item and a subface item on the same coarse array
    items = [_item(subface=-1, coarse_offset=0, fine_offset=0), _item(subface=2, coarse_offset=0, fine_offset=9 * arr)]
    st, _ = _create(items, U=U, cl=arr, fl=10 * arr)
    assert st == 1
    # sharing a coarse array with a different face
    items = [_item(subface=0, coarse_offset=0, fine_offset=0), _item(face=1, subface=1, coarse_offset=0, fine_offset=arr)]
    st, _ = _create(items, U=U, cl=arr, fl=2 * arr)
    assert st == 1
    # partially overlapping coarse arrays
    items = [_item(subface=0, coarse_offset=0, fine_offset=0), _item(subface=1, coarse_offset=arr // 2, fine_offset=arr)]
    st, _ = _create(items, U=U, cl=2 * arr, fl=2 * arr)
    assert st == 1


def test_deep_overlap_needs_factorised_kernels(lib):
    """Overlaps 4 and 5 are served by the factorised kernels only: a plan that
    routes them to the sparse-row kernels is refused on the host."""
    st, h = _create([_item(overlap=4, patch_size=12)], flags=B.FLAG_CSR)
    assert st == 2 and h.value is None
    st, h = _create([_item(overlap=5, patch_size=9, order=1)], flags=B.FLAG_CSR)
    assert st == 2 and h.value is None
