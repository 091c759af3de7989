"""The C-ABI library loads on a machine without a GPU and exports every entry point the header declares.
No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2607_16906_b300", "libhelm.so")


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"HELM_API\s+[\w\s\*]+?\b(helm_\w+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("helm_create", "helm_destroy", "helm_apply", "helm_apply_adjoint", "helm_precond_apply",
              "helm_fgmres_solve", "helm_train_step", "helm_unet_create", "helm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(LIB):
        from paper_2607_16906_b300 import build
        build.build()
    lib = ctypes.CDLL(LIB)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2607_16906_b300 import helm
    assert _declared() <= set(helm.EXPORTED)


def test_param_count_query_needs_no_gpu():
    from paper_2607_16906_b300 import helm
    assert helm.helm_unet_param_count() == 482050
    layers = helm.helm_unet_layers()
    assert layers[0] == (3, 16, 0) and layers[-1] == (16, 2, 2)


def test_argument_errors_are_reported_without_a_gpu():
    """Host-side validation: bad arguments come back as HELM_ERR_INVALID_ARG with a message for the
    calling thread, before anything touches a device."""
    from paper_2607_16906_b300 import helm
    lib = helm._lib
    c_in, c_out, kind = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib.helm_unet_layer(99, ctypes.byref(c_in), ctypes.byref(c_out), ctypes.byref(kind)) == \
        helm.HELM_ERR_INVALID_ARG
    assert b"helm_unet_layer" in lib.helm_last_error()
    w = (ctypes.c_double * 10)()
    h = ctypes.c_void_p()
    assert lib.helm_unet_create(ctypes.byref(h), w, 10) == helm.HELM_ERR_INVALID_ARG  # wrong count
    assert b"expected 482050" in lib.helm_last_error()
    assert lib.helm_apply(None, None, None, 0, 1, None) == helm.HELM_ERR_INVALID_ARG
    assert lib.helm_fgmres_solve(None, None, None, None, 1, None, None, None) == helm.HELM_ERR_INVALID_ARG
    assert lib.helm_tuned_tiles(None, 4) == 0


def test_network_kinds_share_the_generator_layout():
    """The binding's parameter layout of network kind 1 is the oracle's, and the library agrees on the count."""
    from oracle import unet_paper as up
    from paper_2607_16906_b300 import helm
    assert helm.paper_weight_segments() == up.param_segments()
    assert helm._lib.helm_unet_param_count_kind(1) == up.param_count() == 665930
    assert helm._lib.helm_unet_param_count_kind(0) == 482050
    assert helm._lib.helm_unet_param_count_kind(7) == 0
