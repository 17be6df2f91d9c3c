"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/osvmp2.h declares, and its host-only fragment enumeration agrees
bit for bit with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    h = open(os.path.join(ROOT, "include", "osvmp2.h")).read()
    return sorted(set(re.findall(r"\b(osvmp2_[A-Za-z0-9_]+)\s*\(", h)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_16575_gb300 import osvmp2
    if not os.path.exists(osvmp2.LIB_PATH):
        from paper_2603_16575_gb300.build import build
        build()
    return osvmp2.lib()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    from paper_2603_16575_gb300 import osvmp2
    assert set(names) == set(osvmp2.SIGNATURES)


def test_default_opts(lib):
    from paper_2603_16575_gb300 import osvmp2
    o = osvmp2.default_opts()
    assert o.tau_s == 1e-10 and o.max_iter == 100 and o.tol_update == 1e-7


@pytest.mark.parametrize("seed,n,r2,r3", [(0, 40, 8.0, 6.0), (1, 64, 6.0, 4.5), (2, 30, 5.0, 6.0)])
def test_fragment_enumeration_matches_oracle(lib, seed, n, r2, r3):
    from paper_2603_16575_gb300 import osvmp2
    s = synth.make_system(n, 4, 4, seed=seed)
    orbs, w = osvmp2.mbe3_fragments(s.r_occ, r2, r3)
    ref = oracle.mbe3_fragments(s.r_occ, r2, r3)
    assert len(ref) == len(orbs)
    for (o_ref, c_ref), o, c in zip(ref, orbs, w):
        assert tuple(int(x) for x in o if x >= 0) == o_ref
        assert int(c) == c_ref


def test_fragment_enumeration_chain_ties(lib):
    from paper_2603_16575_gb300 import osvmp2
    r = np.zeros((60, 3))
    r[:, 0] = 1.5 * np.arange(60)
    orbs, w = osvmp2.mbe3_fragments(r, 8.0, 6.0)
    ref = oracle.mbe3_fragments(r, 8.0, 6.0)
    assert [tuple(int(x) for x in o if x >= 0) for o in orbs] == [o for o, _ in ref]
    assert [int(x) for x in w] == [c for _, c in ref]


def test_bad_arguments_are_rejected(lib):
    n = ctypes.c_int64(0)
    assert lib.osvmp2_mbe3_fragments(None, 3, 1.0, 1.0, 0, None, None, ctypes.byref(n)) == 1
    assert lib.osvmp2_create(None, 0, None, None) == 1


def test_status_codes_match_the_header(lib):
    """The binding's status table is the header's enum (E_TIMEOUT included), and the
    options struct has the header's size (56 bytes)."""
    from paper_2603_16575_gb300 import osvmp2
    h = open(os.path.join(ROOT, "include", "osvmp2.h")).read()
    enum = dict((name, int(v)) for name, v in re.findall(r"OSVMP2_(OK|E_[A-Z]+)\s*=\s*(\d+)", h))
    assert enum["E_TIMEOUT"] == 7
    assert {v: k for k, v in enum.items()} == osvmp2.STATUS
    assert ctypes.sizeof(osvmp2.Opts) == 56
    o = osvmp2.default_opts()
    assert o.mem_cap_mib == 0
