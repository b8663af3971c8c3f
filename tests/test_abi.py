"""CPU checks of the C-ABI library: it loads, exports every symbol that
include/phix.h declares, and its host-side tables (Leja points, divided
differences) agree with the oracle.  No compute call needs a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_2211_08948_gb300 import build, phix
    build.build()
    return phix, phix.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "phix.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(phix_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_expected_entry_points():
    syms = declared_symbols()
    for s in ["phix_phi_action", "phix_phi_combination", "phix_exprb43_step", "phix_epirk4s3_step",
              "phix_spectrum", "phix_create", "phix_destroy"]:
        assert s in syms


def test_library_exports_every_declared_symbol():
    phix, lib = _lib()
    for s in declared_symbols():
        assert hasattr(lib, s), s
        assert s in phix.EXPORTS, s


def test_version_and_opts_defaults():
    phix, lib = _lib()
    assert phix.phix_version() == 103
    assert lib.phix_opts_size() == ctypes.sizeof(phix.phix_opts)
    assert lib.phix_stats_size() == ctypes.sizeof(phix.phix_stats)
    o = phix.phix_opts_default()
    assert o.prec == phix.PHIX_DF64 and o.m_max == 500 and o.m_min == 3
    assert o.safety == 1.2 and o.rho_re < 0 and o.gamma_cap == 200.0
    assert (o.kiops_m_init, o.kiops_m_max, o.kiops_m_step, o.kiops_max_substeps) == (16, 64, 8, 10000)
    assert o.profile == 0 and o.kernel == phix.PHIX_KERNEL_AUTO
    # the last field: its default read back through the ctypes mirror checks the
    # mirror's layout against the C struct that phix_opts_default fills
    assert o.kiops_fused == 1 and o.chain == phix.PHIX_CHAIN_AUTO and o.jv == 0 and o.leja_augmented == 0
    assert ctypes.sizeof(phix.phix_jop) == 4 * 3 + 4 + 8 * 8 + 8


def test_create_rejects_null():
    phix, lib = _lib()
    assert lib.phix_create(None, None) == phix.PHIX_EINVAL
    assert lib.phix_leja_points(None, 4) == phix.PHIX_EINVAL
    assert lib.phix_destroy(None) == phix.PHIX_EINVAL


def test_host_leja_points_match_oracle():
    from oracle import leja
    phix, _ = _lib()
    a = np.array(phix.phix_leja_points(300))
    b = leja.leja_points(300)
    assert np.max(np.abs(a - b)) < 1e-13


@pytest.mark.parametrize("l,a,b", [(0, -120.0, 60.0), (1, -50.0, 25.0), (3, -3.0, 1.5), (4, -400.0, 200.0)])
def test_host_divided_differences_match_oracle(l, a, b):
    from oracle import leja
    phix, _ = _lib()
    d = np.array(phix.phix_divided_differences(l, a, b, 150))
    x = leja.leja_points(150)
    do = leja.phi_coefficients(x, l, 1.0, a, b)
    # weighted by the Newton basis size on [-2, 2], the tables agree to rounding
    t = np.linspace(-2, 2, 2001)
    w = np.ones_like(t)
    for m in range(150):
        assert abs(d[m] - do[m]) * np.max(np.abs(w)) <= 1e-13 * max(1.0, abs(do[0]))
        w = w * (t - x[m])


@pytest.mark.parametrize("l,a,b", [(1, -50.0, 25.0), (4, -400.0, 200.0)])
def test_host_divided_differences_prefix_is_exact(l, a, b):
    """Tables are built one Leja point at a time; a short table is the prefix
    of a long one bit for bit, so a chain may start on a truncated table and
    continue on the full one with the same coefficients."""
    phix, _ = _lib()
    short = phix.phix_divided_differences(l, a, b, 40)
    full = phix.phix_divided_differences(l, a, b, 300)
    assert short == full[:40]
