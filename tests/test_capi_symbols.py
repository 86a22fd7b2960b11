"""The C-ABI library builds, loads and exports every symbol include/hers.h declares.

CPU only: no compute call is made (there may be no GPU here).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "hers.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hers_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libhers():
    import paper_2003_12197_gb300 as H
    H.build_library()
    return H.lib()


def test_every_declared_symbol_is_exported(libhers):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(libhers, n), n


def test_required_entry_points_declared():
    names = set(declared_functions())
    for n in ("hers_keygen", "hers_encrypt_gallery", "hers_encrypt_probe", "hers_search",
              "hers_decrypt_scores"):
        assert n in names


def test_size_helpers(libhers):
    import paper_2003_12197_gb300 as H
    assert H.hers_ct_bytes() == 2 * 2 * 4096 * 8
    assert H.hers_blocks_for(1) == 1 and H.hers_blocks_for(4096) == 1
    assert H.hers_blocks_for(4097) == 2 and H.hers_blocks_for(100_000_000) == 24415
    # resident gallery: 2 polys x 8 limbs x N int32 per (block, dimension)
    assert H.hers_gallery_bytes(256, 64) == 256 * 64 * 2 * 8 * 4096 * 4
    assert H.hers_probe_bytes(64) == 64 * 2 * 8 * 4096 * 4


def test_status_strings_and_param_check(libhers):
    assert libhers.hers_status_string(0) == b"HERS_OK"
    assert libhers.hers_status_string(-5) == b"HERS_E_PARAM"
    import paper_2003_12197_gb300 as H

    class P(ctypes.Structure):
        _fields_ = [("n", ctypes.c_uint32), ("q", ctypes.c_uint64 * 2), ("t", ctypes.c_uint64),
                    ("flags", ctypes.c_uint32)]
    p = P()
    assert libhers.hers_default_params(ctypes.byref(p)) == 0
    assert p.n == 4096 and p.t == 4169729
    assert p.q[0] == 18014398509309953 and p.q[1] == 18014398509293569
    p.t = 65537    # a prime t that is not = 1 (mod 2N): no plaintext NTT, not supported
    h = ctypes.c_void_p()
    assert libhers.hers_create(ctypes.byref(p), 0, ctypes.byref(h)) == -5
    assert libhers.hers_keygen(None, 1, ctypes.byref(h)) == -1


def test_generated_constants_are_current():
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "paper_2003_12197_gb300", "csrc",
                                                     "gen_consts.py"), "--check"])
    assert r.returncode == 0
    r = subprocess.run([sys.executable, os.path.join(ROOT, "oracle", "gen_cdt.py"), "--check"])
    assert r.returncode == 0


def test_chi_tables_agree_between_library_and_oracle():
    """The two sides derive the chi table by different exact methods: same integers."""
    lib_h = open(os.path.join(ROOT, "paper_2003_12197_gb300", "csrc", "hers_consts.h")).read()
    orc_h = open(os.path.join(ROOT, "oracle", "cdt_table.h")).read()
    lib_t = re.findall(r"(\d+)ULL", lib_h[lib_h.index("HERS_CHI_CDT_INIT"):].split("\n")[0])
    orc_t = re.findall(r"(\d+)ULL", orc_h[orc_h.index("{"):orc_h.index("}")])
    assert lib_t == orc_t and len(lib_t) == 38
