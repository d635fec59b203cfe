"""CPU checks of the C ABI: the library builds, loads, exports every function
include/fabm.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_1710_01133_gb300 as fabm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fabm_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_exports_every_declared_function():
    lib = fabm.load()
    declared = _declared()
    assert {"fabm_create", "fabm_solve", "fabm_solve_batch", "fabm_destroy",
            "fabm_last_error"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(fabm._EXPORTS) == declared


def test_library_links_cuda_runtime_dynamically():
    lib = fabm.load()
    assert os.path.exists(fabm.library_path())
    assert isinstance(lib, ctypes.CDLL)


@pytest.mark.parametrize("kw,msg", [
    (dict(alpha=2.0), "alpha"),
    (dict(alpha=0.0), "alpha"),
    (dict(h=-1.0), "h"),
    (dict(N=0), "N"),
    (dict(dim=2), "dim"),                # lorenz needs dim 3
    (dict(rhs=99), "rhs_id"),
    (dict(params=[10.0, 28.0]), "params"),
    (dict(precision=7), "precision"),
])
def test_create_rejects_bad_arguments(kw, msg):
    args = dict(dim=3, alpha=0.9, h=1e-3, N=100, rhs=fabm.RHS["lorenz"],
                params=[10.0, 28.0, 8.0 / 3.0], precision=fabm.FABM_FP64)
    args.update(kw)
    with pytest.raises(fabm.FabmError) as ei:
        fabm.fabm_create(args["dim"], args["alpha"], args["h"], args["N"], args["rhs"],
                         args["params"], args["precision"])
    assert ei.value.status == fabm.FABM_EINVAL
    assert msg in str(ei.value)


def test_null_handles_are_rejected_or_ignored():
    lib = fabm.load()
    assert lib.fabm_destroy(None) == fabm.FABM_OK
    assert lib.fabm_solve(None, None, None) == fabm.FABM_EINVAL
    assert lib.fabm_set_block(None, 32) == fabm.FABM_EINVAL
    assert lib.fabm_get_block(None) == 0
    assert lib.fabm_set_recurrence_layout(None, 1) == fabm.FABM_EINVAL
    assert lib.fabm_get_recurrence_layout(None) == -1
