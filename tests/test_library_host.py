"""Host-side checks of libhg that need no GPU: it builds, loads, exports every
entry point of include/hg.h, and its pattern table agrees with the oracle's
independently written one."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib(native_cpu):
    import importlib.util

    spec = importlib.util.spec_from_file_location(
        "_hg_build", os.path.join(ROOT, "paper_2504_02271_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_2504_02271_gb300 as hg

    return hg


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "hg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hg_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_entry_points()
    assert "hg_load_csr" in names and "hg_count_patterns" in names
    so = ctypes.CDLL(lib.hg.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert set(names) <= set(lib.hg.EXPORTED)


def test_pattern_table_matches_oracle(lib):
    import oracle

    lut = lib.hg_pattern_table()
    assert [int(x) for x in lut] == [oracle.pattern_of_mask(m) for m in range(128)]


def test_canonical_masks_match_oracle(lib):
    # both sides fold labelled masks into the same canonical forms, written apart
    import oracle

    canon = lib.hg_canonical_masks()
    assert [int(x) for x in canon] == [oracle.canonical_mask(m) for m in range(128)]
    lut = lib.hg_pattern_table()
    # a pattern is one orbit: masks share a pattern iff they share a canonical form
    for a in range(128):
        for b in range(128):
            if lut[a] and lut[b]:
                assert (lut[a] == lut[b]) == (canon[a] == canon[b]), (a, b)


def test_status_strings(lib):
    for s in range(14):
        assert lib.hg_status_str(s) not in ("", "unknown status")
    assert lib.hg_status_str(99) == "unknown status"


def test_no_cpu_fallback_without_gpu(lib):
    import numpy as np
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.HgError) as e:
        lib.hg_load_csr(3, 1, np.array([0, 2]), np.array([0, 1]), stream=0)
    assert e.value.name == "HG_ERR_NO_DEVICE"


def test_concat_members_layout(lib):
    # the binding's concatenation of member CSRs for hg_load_batch: row pointers shifted
    # by the incidences before each member, ids left member-local, empty members kept
    import numpy as np

    from conftest import csr_of

    members = [(3, *csr_of([[0, 1], [1, 2]])),
               (4, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32)),
               (2, *csr_of([[0, 1]]))]
    nv, eoff, eptr, evtx = lib.concat_members(members)
    assert nv.tolist() == [3, 4, 2] and eoff.tolist() == [0, 2, 2, 3]
    assert eptr.tolist() == [0, 2, 4, 6] and evtx.tolist() == [0, 1, 1, 2, 0, 1]


def test_server_and_batch_structs_match_the_header(lib):
    # ctypes layouts of the structs the C ABI exchanges, against sizes from a C compile
    import ctypes
    import subprocess
    import tempfile

    src = ('#include <stdio.h>\n#include "hg.h"\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n",'
           'sizeof(hg_result),sizeof(hg_query),sizeof(hg_server_options),sizeof(hg_server_stats),'
           'sizeof(hg_close_stats),sizeof(hg_tuning),sizeof(hg_autotune_result));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        with open(c, "w") as f:
            f.write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        want = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    hg = lib.hg
    got = [ctypes.sizeof(t) for t in (hg._Result, hg._Query, hg._ServerOptions, hg._ServerStats,
                                      hg._CloseStats, hg._Tuning, hg._AutotuneResult)]
    assert got == want


def test_owner_entry_points_reject_bad_arguments(lib):
    # argument checks come before any device work, so they run without a GPU
    import numpy as np

    so = ctypes.CDLL(lib.hg.LIB_PATH)
    counts = np.zeros(21, dtype=np.uint64)
    owners = np.zeros(4, dtype=np.int32)
    vp = ctypes.c_void_p
    so.hg_count_owned.argtypes = [vp, vp, ctypes.c_int32, vp, vp]
    so.hg_out_degrees.argtypes = [vp, vp]
    invalid = {name: code for code, name in lib.hg.STATUS.items()}["HG_ERR_INVALID_ARG"]
    assert so.hg_count_owned(None, owners.ctypes.data, 4, counts.ctypes.data, None) == invalid
    assert so.hg_out_degrees(None, owners.ctypes.data) == invalid
