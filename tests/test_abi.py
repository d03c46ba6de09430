"""Host-only checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects bad arguments before touching the device."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_1804_06231_gb300 import build, pv
    build.build_library()
    return pv.load_library()


def header_functions():
    src = (ROOT / "include" / "pv.h").read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pv_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    from paper_1804_06231_gb300 import pv
    names = header_functions()
    assert set(names) == set(pv.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    from paper_1804_06231_gb300 import pv
    for code in range(8):
        s = pv.pv_status_str(code)
        assert s and s != "unknown status"
    assert pv.pv_status_str(99) == "unknown status"


def test_struct_layout_matches_header():
    """ctypes mirrors of the public structs have the C layout (x86-64/aarch64 LP64)."""
    from paper_1804_06231_gb300 import pv
    assert ctypes.sizeof(pv.pv_box_desc) == 32
    assert pv.pv_box_desc.nc.offset == 24
    assert ctypes.sizeof(pv.pv_grid_desc) == 32
    assert ctypes.sizeof(pv.pv_stats) == 144
    assert ctypes.sizeof(pv.pv_tuning) == 32


def test_argument_errors_return_before_device_work(lib):
    from paper_1804_06231_gb300 import pv
    out = ctypes.c_void_p()
    assert lib.pv_grid_create(None, ctypes.byref(out)) == 1
    boxes = (pv.pv_box_desc * 1)(pv.pv_box_desc(0, 10, 1.0, 2))
    desc = pv.pv_grid_desc(1, boxes, 0.0, 0)
    assert lib.pv_grid_create(ctypes.byref(desc), ctypes.byref(out)) == 2   # nc < 3
    boxes = (pv.pv_box_desc * 2)(pv.pv_box_desc(0, 10, 1.0, 3), pv.pv_box_desc(5, 10, 1.0, 3))
    desc = pv.pv_grid_desc(2, boxes, 0.0, 0)
    assert lib.pv_grid_create(ctypes.byref(desc), ctypes.byref(out)) == 1   # not contiguous
    boxes = (pv.pv_box_desc * 1)(pv.pv_box_desc(0, 10, -1.0, 3))
    desc = pv.pv_grid_desc(1, boxes, 0.0, 0)
    assert lib.pv_grid_create(ctypes.byref(desc), ctypes.byref(out)) == 1   # L <= 0
    desc = pv.pv_grid_desc(1, boxes, 0.0, 7)
    assert lib.pv_grid_create(ctypes.byref(desc), ctypes.byref(out)) == 1   # flags != 0
    assert lib.pv_sort_cells(None, None, None, None, ctypes.c_float(0), None) == 1
    assert lib.pv_density(None, None, None, None, None) == 1
    assert lib.pv_density_symmetric(None, None, None, None, None) == 1
    assert lib.pv_density_backward(None, None, None, None, None, None) == 1
    assert lib.pv_count_candidates(None, None) == 1
    assert lib.pv_grid_sync(None, None) == 1
    assert lib.pv_grid_stats(None, None) == 1
    assert lib.pv_grid_time_sweeps(None, 1) == 1
    assert lib.pv_grid_set_slot_mask(None, 1) == 1
    assert lib.pv_update_positions(None, None, None, None) == 1
    assert lib.pv_raw_interactions(None, 4, None, 4, ctypes.c_float(1.0), 1, None, None) == 1
    assert lib.pv_raw_interactions(None, -1, None, 4, ctypes.c_float(1.0), 1, None, None) == 1
    assert lib.pv_raw_interactions(None, 0, None, 0, ctypes.c_float(0.0), 1, None, None) == 1
    fl = ctypes.c_double(0.0)
    assert lib.pv_fp32_probe(0, 0, None, 256, ctypes.byref(fl), None) == 1      # iters < 1
    assert lib.pv_fp32_probe(0, 10, None, 100, ctypes.byref(fl), None) == 1     # not 256k
    assert lib.pv_fp32_probe(0, 10, None, 256, ctypes.byref(fl), None) == 1     # no sink
    assert lib.pv_fp32_probe(1, 10, None, 256, None, None) == 1                 # no flops
    assert lib.pv_fp32_probe(1, 10, None, 0, ctypes.byref(fl), None) == 0       # nothing queued
    t = pv.pv_tuning(3, 2)
    assert lib.pv_grid_set_tuning(None, ctypes.byref(t)) == 1
    assert lib.pv_grid_get_tuning(None, ctypes.byref(t)) == 1
    assert lib.pv_grid_sweep_times(None, None, None) == 1
    assert lib.pv_grid_destroy(None) == 0


def test_product_path_does_not_import_oracle():
    """The package never imports the oracle (it is test infrastructure)."""
    pkg = ROOT / "paper_1804_06231_gb300"
    for f in list(pkg.glob("*.py")) + list((pkg / "csrc").glob("*")):
        text = f.read_text()
        assert "import oracle" not in text and "from oracle" not in text, f
        assert "pv_oracle" not in text, f


def test_slot_masks_of_classes():
    from paper_1804_06231_gb300 import pv
    masks = [pv.slot_mask_of_class(c) for c in range(4)]
    assert [bin(m).count("1") for m in masks] == [1, 6, 12, 8]
    assert masks[0] == 1 << 13
    assert sum(masks) == pv.SLOT_MASK_ALL
