"""CPU-only checks of the C-ABI library: it builds, loads and exports every
symbol declared in include/*.h, and host-side validation works without a GPU."""
import ctypes
import glob
import os
import re

import pytest

from paper_2112_01508_gb300 import _native as nat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions(header="*.h"):
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", header)):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(p3m_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = nat.load()
    declared = _declared_functions("p3m_sr.h")
    assert declared, "no declarations found"
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    assert set(nat.EXPORTS) == declared


def test_mesh_library_exports_every_declared_symbol():
    lib = nat.load_pm()
    declared = _declared_functions("p3m_pm.h")
    assert declared, "no declarations found"
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    assert set(nat.PM_EXPORTS) == declared
    assert _declared_functions() == declared | set(nat.EXPORTS)


def _pm_params(**kw):
    p = nat.PMParams()
    p.n, p.box, p.n_phi, p.x_s, p.G_m, p.p_i, p.p_d, p.precision = 1000, 1.0, 64, 1.25 / 64, 1e-3, 2, 4, 32
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw", [dict(n=-1), dict(box=0.0), dict(n_phi=7), dict(n_phi=6), dict(n_phi=8192),
                                dict(x_s=-0.1), dict(p_i=0), dict(p_i=5), dict(p_d=3), dict(p_d=10),
                                dict(precision=16), dict(G_m=float("inf"))])
def test_mesh_create_rejects_bad_parameters(kw):
    # validation happens before any device call, so this runs without a GPU
    st, ctx = nat.p3m_pm_create(_pm_params(**kw), 0)
    assert st == nat.P3M_ERR_INVALID
    assert not ctx.value


def _params(**kw):
    p = nat.P3MParams()
    p.n, p.box, p.x_s, p.x_r, p.G_m = 1000, 1.0, 0.01, 0.045, 1e-3
    p.softening, p.eps, p.n_rung = 2, 1e-3, 8
    p.n_sub[0] = p.n_sub[1] = p.n_sub[2] = 2
    for k, v in kw.items():
        if k == "n_sub":
            p.n_sub[0], p.n_sub[1], p.n_sub[2] = v
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw,status", [
    (dict(x_r=0.3), nat.P3M_ERR_TOO_FEW_TILES),     # floor(1/0.3) = 3 tiles < 4
    (dict(n=-1), nat.P3M_ERR_INVALID),
    (dict(box=0.0), nat.P3M_ERR_INVALID),
    (dict(x_s=-1.0), nat.P3M_ERR_INVALID),
    (dict(softening=3), nat.P3M_ERR_INVALID),
    (dict(eps=0.0), nat.P3M_ERR_INVALID),
    (dict(n_sub=(0, 2, 2)), nat.P3M_ERR_INVALID),
    (dict(n_rung=9), nat.P3M_ERR_INVALID),
    (dict(eps=0.05), nat.P3M_ERR_INVALID),           # softening beyond 2 x_s
])
def test_create_rejects_bad_parameters(kw, status):
    st, ctx = nat.p3m_sr_create(_params(**kw), 0)
    assert st == status
    assert not ctx.value


def test_null_context_is_rejected():
    lib = nat.load()
    assert lib.p3m_sr_sync(None) == nat.P3M_ERR_INVALID
    assert lib.p3m_sr_forces(None, None, 32, None) == nat.P3M_ERR_INVALID
    assert lib.p3m_sr_last_error(None) == b"null context"
    lib.p3m_sr_destroy(None)


def test_header_documents_every_entry_point():
    text = open(os.path.join(ROOT, "include", "p3m_sr.h")).read()
    for name in nat.EXPORTS:
        assert name in text
    assert "Section 2.1.3" in text and "Eq. rung" in text


def _noalloc_params(**kw):
    """32^3-recipe parameters (x_s = 1.25/64, x_r = 4.5 x_s, 11 tiles per dimension)."""
    x_s = 1.25 / 64
    return _params(**{**dict(n=1 << 15, x_s=x_s, x_r=4.5 * x_s, eps=0.03 / 32), **kw})


@pytest.mark.parametrize("kw", [
    dict(n=(1 << 16) + 1),                                     # beyond the particle limit
    dict(n_sub=(6, 6, 6)),                                     # (11 * 6)^3 = 287,496 subtiles > 2^18
    dict(x_r=1.0 / 41.5, x_s=1.0 / 41.5 / 4.5, eps=1e-4, n_sub=(1, 1, 1)),  # 41^2 ceil(41/4) = 18,491 segments > 2^14
    dict(x_s=1.25 / 64 * 0.9),                                 # x_r = 5 x_s: beyond the FP32 erfc fit
    dict(n=-1),
    dict(x_r=0.3),                                             # fewer than 4 tiles
])
def test_forces_noalloc_rejects_inputs_beyond_its_limits(kw):
    # every limit is checked on the host before any device call, so this runs without a GPU
    lib = nat.load()
    p = _noalloc_params(**kw)
    st = lib.p3m_sr_forces_noalloc(ctypes.byref(p), None, None, None)
    assert st in (nat.P3M_ERR_INVALID, nat.P3M_ERR_TOO_FEW_TILES)


def test_forces_noalloc_limits_admit_the_largest_sets():
    # at the limits (n = 2^16, 2^18 subtiles would need n_sub = 5.8; n_sub = 5 gives
    # 166,375) an empty particle set is accepted without touching the device
    lib = nat.load()
    p = _noalloc_params(n=0, n_sub=(5, 5, 5))
    assert lib.p3m_sr_forces_noalloc(ctypes.byref(p), None, None, None) == nat.P3M_OK
