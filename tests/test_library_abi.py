"""CPU checks of the C ABI: the library loads, exports every function that
include/matcha.h declares, and rejects bad arguments on the host before any
device work."""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

import paper_2603_15285_gb300 as m
from paper_2603_15285_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "matcha.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(matcha_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return m.lib()


def test_every_declared_symbol_is_exported(L):
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(m.SYMBOLS) == names


def test_status_strings(L):
    for s in range(6):
        assert L.matcha_status_string(s)
    assert L.matcha_status_string(0) == b"ok"


def _desc(**kw):
    d = m.PlanDesc()
    d.box_n, d.n_shells, d.r_max, d.L0, d.K_oversample, d.P_max, d.M_iter = 32, 12, 0.0, 8, 2, 8, 3
    sched = kw.pop("L_sched", (8, 12, 16))
    d.n_levels = len(sched)
    for i, v in enumerate(sched):
        d.L_sched[i] = v
    d.precision = 0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("bad", [
    dict(box_n=2), dict(n_shells=0), dict(L0=0), dict(K_oversample=17), dict(P_max=0),
    dict(P_max=33), dict(M_iter=0), dict(precision=7), dict(L_sched=(8, 8, 16)),
    dict(L_sched=(4, 12, 16)), dict(r_max=float("nan")), dict(refine=2),
])
def test_plan_create_rejects_bad_descriptors_on_host(L, bad):
    d = _desc(**bad)
    h = ctypes.c_void_p()
    assert L.matcha_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert not h.value


def test_bandwidth_limit_is_unsupported_not_a_crash(L):
    d = _desc(L_sched=(8, 40, 120))
    h = ctypes.c_void_p()
    assert L.matcha_plan_create(ctypes.byref(d), ctypes.byref(h)) == 5


def test_null_handles_are_rejected(L):
    assert L.matcha_plan_create(None, None) == 1
    assert L.matcha_plan_destroy(None) == 0
    assert L.matcha_analyze(None, None, 1, None, None) == 1
    assert L.matcha_align(None, None, None, 1, 1, None, None, None, None, None, None, None, 0, None) == 1


def test_newer_entry_points_check_arguments_on_the_host(L):
    """The gradient, tuning and status calls reject missing handles and
    outputs before any device work (status 1 = MATCHA_ERR_INVALID_ARG)."""
    import ctypes
    sz = ctypes.c_size_t(0)
    bits = ctypes.c_int(0)
    assert L.matcha_template_grad_workspace_size(None, 4, 0, ctypes.byref(sz)) == 1
    assert L.matcha_template_grad(None, None, None, 4, 0, None, None, None, None, None, None,
                                  None, 0, None) == 1
    assert L.matcha_plan_autotune(None, None, None, 4, 1, None, None, 0, None, None) == 1
    assert L.matcha_plan_device_status(None, ctypes.byref(bits)) == 1
    assert L.matcha_plan_set_wait_limit(None, 0) == 1
    assert L.matcha_host_workspace_size(None, 4, 1, ctypes.byref(sz)) == 1


def test_layout_helper_counts_entries():
    for Lj in (8, 16, 32):
        rows = m.corr_layout(Lj)
        used = rows[rows[:, 1] <= rows[:, 0]]
        # every (l, m, n) with m >= |n| once, plus one empty slot per (m, l)
        assert len(used) == sum((l + 1) ** 2 for l in range(Lj + 1))
        assert len(set(map(tuple, used))) == len(used)
        assert len(rows) - len(used) == sum(Lj - mm + 1 for mm in range(Lj + 1))
        assert len(rows) == 2 * sum((mm + 1) * (Lj - mm + 1) for mm in range(Lj + 1))


def test_corr_pairs_deinterleaves_partners():
    # group entry e holds reals 8e + 2k + h: component k of slot h
    n = 6
    raw = np.arange(4 * n, dtype=np.float64).reshape(n, 2, 2)
    rows = m.corr_pairs(raw)
    for e in range(n // 2):
        for h in range(2):
            got = rows[2 * e + h].reshape(4)
            assert list(got) == [8 * e + 2 * k + h for k in range(4)]
    t = torch.arange(4 * n, dtype=torch.float64).reshape(1, n, 2, 2)
    assert np.array_equal(m.corr_pairs(t)[0].numpy(), rows)
