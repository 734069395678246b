"""CPU checks of the C ABI: the library loads, exports every symbol include/progot.h
declares, and its host-only logic (argument checks, schedules, workspace sizing)
behaves; nothing here launches a kernel."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import progot_oracle as O
from paper_2406_05061_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared_functions():
    names = []
    for path in HEADERS:
        with open(path) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for mt in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", text, flags=re.M):
            name = mt.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(native.LIB_PATH):
        from paper_2406_05061_gb300 import build
        build.build()
    return native.lib()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert "progot_solve" in declared and "sinkhorn_potentials" in declared
    bound = {s[0] for s in native.SIGNATURES}
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert name in bound, f"{name} has no ctypes signature in the binding"
    assert bound <= set(declared)


def test_alpha_schedules_match_oracle(lib):
    for K in (1, 2, 3, 4, 8, 16):
        for kind in ("constant", "accelerated", "decelerated"):
            np.testing.assert_allclose(native.progot_schedule_alpha(K, kind), O.alpha_schedule(K, kind), rtol=1e-15)


def test_invalid_arguments_are_rejected_on_the_host(lib):
    fake = ctypes.c_void_p(0x100000)
    ws = ctypes.c_void_p(0x200000)
    # n = 0
    rc = lib.sinkhorn_potentials(fake, None, 0, fake, None, 4, 2, 1.0, 1e-3, 10, 0, fake, fake, 1, None, None,
                                 ws, 1 << 20, None)
    assert rc == native.PROGOT_ERR_INVALID_ARG and "positive" in native.last_error()
    # eps <= 0
    rc = lib.sinkhorn_potentials(fake, None, 4, fake, None, 4, 2, 0.0, 1e-3, 10, 0, fake, fake, 1, None, None,
                                 ws, 1 << 20, None)
    assert rc == native.PROGOT_ERR_INVALID_ARG and "eps" in native.last_error()
    # NULL x
    rc = lib.sinkhorn_potentials(None, None, 4, fake, None, 4, 2, 1.0, 1e-3, 10, 0, fake, fake, 1, None, None,
                                 ws, 1 << 20, None)
    assert rc == native.PROGOT_ERR_INVALID_ARG
    # unknown precision
    rc = lib.sinkhorn_potentials(fake, None, 4, fake, None, 4, 2, 1.0, 1e-3, 10, 9, fake, fake, 1, None, None,
                                 ws, 1 << 20, None)
    assert rc == native.PROGOT_ERR_INVALID_ARG and "precision" in native.last_error()
    # workspace NULL, misaligned, too small
    rc = lib.sinkhorn_potentials(fake, None, 4, fake, None, 4, 2, 1.0, 1e-3, 10, 0, fake, fake, 1, None, None,
                                 None, 0, None)
    assert rc == native.PROGOT_ERR_WORKSPACE
    rc = lib.sinkhorn_potentials(fake, None, 4, fake, None, 4, 2, 1.0, 1e-3, 10, 0, fake, fake, 1, None, None,
                                 ctypes.c_void_p(0x200010), 1 << 20, None)
    assert rc == native.PROGOT_ERR_WORKSPACE and "aligned" in native.last_error()
    rc = lib.sinkhorn_potentials(fake, None, 4, fake, None, 4, 2, 1.0, 1e-3, 10, 0, fake, fake, 1, None, None,
                                 ws, 16, None)
    assert rc == native.PROGOT_ERR_WORKSPACE and "needed" in native.last_error()


def test_progot_solve_rejects_bad_schedules(lib):
    fake = ctypes.c_void_p(0x100000)
    K = 2
    for alpha, eps, tau in (([0.5, 1.5], [1.0, 1.0], [1e-3, 1e-3]), ([0.5, 1.0], [1.0, -1.0], [1e-3, 1e-3]),
                            ([0.0, 1.0], [1.0, 1.0], [1e-3, 1e-3]), ([0.5, 1.0], [1.0, 1.0], [1e-3, -1.0])):
        a_h = np.asarray(alpha, dtype=np.float64)
        e_h = np.asarray(eps, dtype=np.float64)
        t_h = np.asarray(tau, dtype=np.float64)
        rc = lib.progot_solve(fake, None, 8, fake, None, 8, 2, K, a_h.ctypes.data_as(ctypes.c_void_p),
                              e_h.ctypes.data_as(ctypes.c_void_p), t_h.ctypes.data_as(ctypes.c_void_p), 10, 0,
                              fake, fake, None, None, None, None, ctypes.c_void_p(0x200000), 1 << 20, None)
        assert rc == native.PROGOT_ERR_INVALID_ARG


def test_workspace_size_is_linear_in_problem_size(lib):
    s1 = native.workspace_size(8192, 8192, 64)
    s2 = native.workspace_size(65536, 65536, 64)
    assert 0 < s1 < s2 < 16 * s1
    assert native.workspace_size(0, 10, 2) == 0
    assert native.workspace_size(8192, 8192, 256) > s1


def test_binding_refuses_non_cuda_tensors(lib):
    torch = pytest.importorskip("torch")
    x = torch.zeros(4, 2)
    with pytest.raises(TypeError):
        native.sinkhorn_potentials(x, x, 1.0, 1e-3)


def test_tau_schedule_matches_oracle(lib):
    for K in (1, 2, 5, 16):
        np.testing.assert_allclose(native.progot_schedule_tau(K, 0.01, 1e-3), O.tau_schedule(K, 0.01, 1e-3),
                                   rtol=1e-14)
    out = np.zeros(3)
    assert lib.progot_schedule_tau(3, -1.0, 1e-3, out.ctypes.data_as(ctypes.c_void_p)) == native.PROGOT_ERR_INVALID_ARG


def test_widened_entry_points_check_arguments_on_the_host(lib):
    fake = ctypes.c_void_p(0x100000)
    ws = ctypes.c_void_p(0x200000)
    h = np.ones(2, dtype=np.float64)
    hp = h.ctypes.data_as(ctypes.c_void_p)
    # theta <= 0, missing eps_out
    rc = lib.progot_solve_theta(fake, None, 8, fake, None, 8, 2, 2, hp, 0.0, hp, 10, 0, fake, fake, None, None,
                                None, None, hp, ws, 1 << 20, None)
    assert rc == native.PROGOT_ERR_INVALID_ARG and "theta" in native.last_error()
    rc = lib.progot_solve_theta(fake, None, 8, fake, None, 8, 2, 2, hp, 0.1, hp, 10, 0, fake, fake, None, None,
                                None, None, None, ws, 1 << 20, None)
    assert rc == native.PROGOT_ERR_INVALID_ARG
    met = native.CouplingMetricsStruct()
    rc = lib.coupling_metrics(fake, None, 8, fake, None, 8, 2, fake, fake, None, -1.0, ctypes.byref(met), ws, 1 << 20,
                              None)
    assert rc == native.PROGOT_ERR_INVALID_ARG and "eps" in native.last_error()
    rc = lib.coupling_metrics(fake, None, 8, fake, None, 8, 2, None, fake, None, 1.0, ctypes.byref(met), ws, 1 << 20,
                              None)
    assert rc == native.PROGOT_ERR_INVALID_ARG
    val = ctypes.c_double(0.0)
    rc = lib.sinkhorn_divergence(fake, None, 8, fake, None, 8, 2, 1.0, -1.0, 10, 0, ctypes.byref(val), None, None,
                                 ws, 1 << 20, None)
    assert rc == native.PROGOT_ERR_INVALID_ARG and "tau" in native.last_error()
    rc = lib.sinkhorn_divergence(fake, None, 8, fake, None, 8, 2, 1.0, 1e-3, 10, 0, ctypes.byref(val), None, None,
                                 ws, 16, None)
    assert rc == native.PROGOT_ERR_WORKSPACE
    rc = lib.coupling_diagonal(fake, fake, 8, 2, fake, fake, 0.0, None, None, None, ws, 1 << 20, None)
    assert rc == native.PROGOT_ERR_INVALID_ARG


def test_pnorm_entry_points_check_p_on_the_host(lib):
    fake = ctypes.c_void_p(0x100000)
    ws = ctypes.c_void_p(0x200000)
    for p in (1.0, 0.5, -2.0, 9.0, float("nan")):
        rc = lib.sinkhorn_potentials_pnorm(fake, None, 8, fake, None, 8, 2, p, 1.0, 1e-3, 10, fake, fake, 1, None,
                                           None, ws, 1 << 20, None)
        assert rc == native.PROGOT_ERR_INVALID_ARG and "p" in native.last_error()
    out = ctypes.c_double(0.0)
    assert lib.progot_mean_cost_pnorm(fake, 8, fake, 8, 2, 1.0, ctypes.byref(out), ws, 1 << 20,
                                      None) == native.PROGOT_ERR_INVALID_ARG
    h = np.ones(2, dtype=np.float64)
    hp = h.ctypes.data_as(ctypes.c_void_p)
    # no eps schedule and no theta
    rc = lib.progot_solve_pnorm(fake, None, 8, fake, None, 8, 2, 1.5, 2, hp, None, 0.0, hp, 10, fake, fake, None,
                                None, None, None, None, ws, 1 << 20, None)
    assert rc == native.PROGOT_ERR_INVALID_ARG and "theta" in native.last_error()
