"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/hetal.h declares (no compute call here)."""
import ctypes
import subprocess

import pytest

from paper_2403_14111_gb300 import build as gbuild
import paper_2403_14111_gb300.hetal as H


@pytest.fixture(scope="module")
def libpath():
    return gbuild.build()


def test_exports_every_declared_symbol(libpath):
    names = H.declared_symbols()
    assert len(names) >= 40
    L = ctypes.CDLL(libpath)
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln and ln.split()[-1].startswith("hetal_")}
    assert exported == set(names)


def test_binding_covers_header(libpath):
    assert set(H._SIGS) == set(H.declared_symbols())
    H.lib()


def test_null_arguments_are_rejected_without_a_gpu(libpath):
    L = H.lib()
    assert L.hetal_ctx_create(None, 0, None, None) == H.ERR_INVALID_ARG
    assert L.hetal_ptset_put(None, 1, 0, 0, None, 0) == H.ERR_INVALID_ARG
    assert L.hetal_mat_desc_get(None, None) == H.ERR_INVALID_ARG
    L.hetal_mat_free(None)
    L.hetal_ctx_destroy(None)
    # graph recording: handles checked before any device work
    assert L.hetal_graph_begin(None) == H.ERR_INVALID_ARG
    assert L.hetal_graph_end(None, None) == H.ERR_INVALID_ARG
    assert L.hetal_graph_launch(None, None) == H.ERR_INVALID_ARG
    n = ctypes.c_longlong(-1)
    assert L.hetal_graph_kernels(None, ctypes.byref(n)) == H.ERR_INVALID_ARG and n.value == -1
    L.hetal_graph_free(None)
    rate = ctypes.c_double()
    assert L.hetal_probe_mac_rate(None, 100, ctypes.byref(rate)) == H.ERR_INVALID_ARG


def test_ptset_roundtrip_host_only(libpath):
    import numpy as np
    s = H.hetal_ptset_create()
    H.hetal_ptset_put(s, H.PT_DMASK, 3, 2, np.arange(16))
    H.hetal_ptset_free(s)
