"""The C ABI on the host: libitp.so loads and exports every entry point that
include/itp.h declares, the binding declares each of them, and argument
checks that need no GPU reject bad input.  No compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "itp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(itp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("itp_create_grid", "itp_set_potential", "itp_propagate", "itp_orthonormalize",
              "itp_energies", "itp_set_states", "itp_get_states", "itp_destroy",
              "itp_last_error", "itp_polish"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_0809_3739_gb300 import itp
    lib = ctypes.CDLL(itp.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    bound = {s[0] for s in itp.SIGNATURES}
    assert set(_declared()) == bound


def test_bad_grid_rejected_before_any_device_call():
    import paper_0809_3739_gb300 as P
    for dims in ((33, 32, 32), (32, 32, 512), (54, 32, 32), (0, 8, 8)):
        with pytest.raises(P.ItpError) as ei:
            P.ItpGrid(*dims, 10.0, 10.0, 10.0, 4)
        assert ei.value.code == 1
        assert "unsupported grid" in P.itp_last_error(None)
    with pytest.raises(P.ItpError) as ei:
        P.ItpGrid(32, 32, 32, 10.0, 10.0, 10.0, 257)
    assert ei.value.code == 1


def test_supported_sizes_agree_with_input_module():
    """The grid edges the library plans for are the ones itp_workloads calls
    supported (checked through the library's own argument check)."""
    import paper_0809_3739_gb300 as P
    from itp_workloads import supported_dim
    for n in range(2, 260, 2):
        try:
            P.ItpGrid(n, 8, 8, 10.0, 10.0, 10.0, 1).close()
            ok = True
        except P.ItpError as e:
            ok = e.code != 1
        assert ok == supported_dim(n), n
