"""CPU tests of the C ABI: the library loads, exports every declared symbol,
and its host-side validation and planning behave (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from synthetic import robots as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_05493_gb300 import build
    build()
    from paper_2603_05493_gb300 import _lib
    return _lib


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wbe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wb_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    L = lib.load()
    names = declared_functions()
    assert "wb_eval" in names and "wb_eval_backward" in names and "wb_load_robot" in names
    for name in names:
        assert hasattr(L, name), name
    assert set(names) <= set(lib.SIGNATURES), set(names) - set(lib.SIGNATURES)
    assert L.wb_version() >= 100


def test_plan_counts(lib):
    from paper_2603_05493_gb300 import wbe
    info, rounds = wbe.plan_info(R.r48())
    assert info["n_links"] == 49 and info["dof"] == 48
    assert info["n_spheres"] == 200 and info["n_pairs"] == 15392
    assert info["n_levels"] == 13 and info["max_level_width"] == 6
    assert info["n_pair_blocks"] == 962
    # every lane of a 32-lane group gets ceil(962 / 32) blocks at most
    assert rounds[3] == 31
    info, rounds = wbe.plan_info(R.r7())
    assert (info["n_pairs"], info["n_pair_blocks"], info["n_levels"]) == (240, 15, 7)
    info, _ = wbe.plan_info(R.mixed_joint_tree())
    assert info["dof"] == 5


def _plan(desc):
    from paper_2603_05493_gb300 import wbe
    return wbe.plan_info(desc)


def _code(desc):
    from paper_2603_05493_gb300 import _lib
    try:
        _plan(desc)
        return 0
    except _lib.WbError as e:
        return e.code


def test_validation_errors(lib):
    L = lib
    base = R.r7()
    import dataclasses as dc

    bad = dc.replace(base, parent=np.array([-1, 0, 3, 2, 3, 4, 5], np.int32))
    assert _code(bad) == L.WB_ETOPO
    bad = dc.replace(base, jtype=np.array([1, 1, 5, 1, 1, 1, 1], np.int32))
    assert _code(bad) == L.WB_ETOPO
    ax = base.axis.copy()
    ax[3] *= 1.1
    assert _code(dc.replace(base, axis=ax)) == L.WB_EINVAL
    T = base.T_fixed.copy()
    T[2, 0] = 2.0
    assert _code(dc.replace(base, T_fixed=T)) == L.WB_EINVAL
    jidx = base.jidx.copy()
    jidx[6] = 9  # joints 7, 8 drive nothing
    assert _code(dc.replace(base, jidx=jidx)) == L.WB_ETOPO
    assert _code(base.with_pairs([[0, 100]])) == L.WB_ERANGE
    assert _code(base.with_pairs([[5, 5]])) == L.WB_ERANGE
    assert _code(base.with_pairs([[1, 9], [1, 9]])) == L.WB_ERANGE
    sl = base.sph_link.copy()
    sl[0] = 7
    assert _code(dc.replace(base, sph_link=sl)) == L.WB_ERANGE
    assert _code(base.with_point_masses([7], [1.0], [[0, 0, 0]])) == L.WB_ERANGE
    m = base.mass.copy()
    m[0] = -1
    assert _code(dc.replace(base, mass=m)) == L.WB_EINVAL
    # too many links
    n = 300
    big = R._plain("big", [-1] + list(range(n - 1)), [1] * n, [[0, 0, 1]] * n,
                   [R._Tp(0.1, 0, 0)] * n, [1.0] * n, np.zeros((n, 3)),
                   [[0.1, 0.1, 0.1, 0, 0, 0]] * n, [0], [[0, 0, 0]], [0.1])
    assert _code(big) == L.WB_ETOOBIG


def test_unordered_pairs_are_sorted(lib):
    from paper_2603_05493_gb300 import wbe
    base = R.r23()
    perm = np.random.default_rng(0).permutation(base.P)
    info, _ = wbe.plan_info(base.with_pairs(base.pairs[perm]))
    assert info["n_pairs"] == base.P


def test_no_pairs_and_no_spheres_plan(lib):
    from paper_2603_05493_gb300 import wbe
    info, rounds = wbe.plan_info(R.r7().with_pairs(np.zeros((0, 2), np.int32)))
    assert info["n_pairs"] == 0 and info["n_pair_blocks"] == 0 and rounds == [0, 0, 0, 0]


def test_load_on_missing_device_reports_edevice(lib):
    from paper_2603_05493_gb300 import wbe
    L = lib.load()
    keep = []
    tree, sph, pairs, inert = wbe.descriptors(R.r7(), keep)
    h = C.c_void_p()
    rc = L.wb_load_robot(C.byref(tree), C.byref(sph), C.byref(pairs), C.byref(inert), 99,
                         C.byref(h))
    assert rc == lib.WB_EDEVICE
    assert b"device" in L.wb_last_error()


def test_size_limits(lib):
    """The largest robot the library takes plans on the host (255 links,
    1020 spheres, 32 levels); one link or one sphere more is WB_ETOOBIG."""
    from dataclasses import replace
    big = R.max_size()
    info, _ = _plan(big)
    assert (info["n_links"], info["n_spheres"], info["n_levels"]) == (255, 1020, 32)
    assert info["n_pairs"] == 330624 and info["n_pair_blocks"] <= 65535
    more_sph = replace(big, sph_link=np.append(big.sph_link, 1),
                       sph_c=np.vstack([big.sph_c, [[0, 0, 0]]]), sph_r=np.append(big.sph_r, 0.01))
    assert _code(more_sph) == lib.WB_ETOOBIG
    more_links = replace(big, parent=np.append(big.parent, 0), jtype=np.append(big.jtype, 1),
                         axis=np.vstack([big.axis, [[0, 0, 1]]]),
                         T_fixed=np.vstack([big.T_fixed, big.T_fixed[1:2]]),
                         jidx=np.append(big.jidx, big.dof), mimic_mult=np.append(big.mimic_mult, 1),
                         mimic_off=np.append(big.mimic_off, 0), mass=np.append(big.mass, 1),
                         com=np.vstack([big.com, [[0, 0, 0]]]),
                         Icom=np.vstack([big.Icom, big.Icom[1:2]]))
    assert _code(more_links) == lib.WB_ETOOBIG
    deep = R.deep_chain(33)  # plans; only the sweep kernels refuse it
    info, _ = _plan(deep)
    assert info["n_levels"] == 33
