"""The C-ABI library builds, loads and exports every symbol the header
declares; struct layouts agree between the header and the Python binding.
No GPU is needed (no compute call is made)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cherenkov.h")


@pytest.fixture(scope="module")
def lib_path():
    from paper_2405_04229_gb300 import build
    return build.build()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(cs_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib_path):
    names = _declared_functions()
    assert len(names) >= 12
    L = C.CDLL(lib_path)
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(r" T %s$" % n, out, flags=re.M), n


def test_struct_layouts_match_binding(lib_path):
    from paper_2405_04229_gb300 import binding as B
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "cherenkov.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(cs_segment), sizeof(cs_record), sizeof(cs_atmosphere_desc),
         sizeof(cs_detector_desc), sizeof(cs_output), sizeof(cs_opts));
  printf("%zu %zu %zu %zu\n", offsetof(cs_atmosphere_desc, table_dh), offsetof(cs_detector_desc, tel_xyzr),
         offsetof(cs_output, record_count), offsetof(cs_opts, blocks_per_sm));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "l")
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe])
        a, b = subprocess.check_output([exe], text=True).strip().split("\n")
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [64, 56, C.sizeof(B.cs_atmosphere_desc), C.sizeof(B.cs_detector_desc), C.sizeof(B.cs_output),
                     C.sizeof(B.cs_opts)]
    assert B.SEGMENT_DTYPE.itemsize == 64 and B.RECORD_DTYPE.itemsize == 56
    assert offs == [B.cs_atmosphere_desc.table_dh.offset, B.cs_detector_desc.tel_xyzr.offset,
                    B.cs_output.record_count.offset, B.cs_opts.blocks_per_sm.offset]


def test_status_strings_and_no_silent_fallback(lib_path):
    from paper_2405_04229_gb300 import binding as B
    assert B.status_string(B.CS_OK) == "CS_OK"
    assert B.status_string(B.CS_ERR_CAPACITY) == "CS_ERR_CAPACITY"
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        # without a GB300 every device call fails loudly; there is no CPU path
        with pytest.raises(B.CSError):
            B.cs_device_sm_count()
        with pytest.raises(B.CSError):
            B.Atmosphere(layered=__import__("paper_2405_04229_gb300.synth", fromlist=["x"]).US_STANDARD)


def test_invalid_descriptors_are_rejected_before_any_device_work(lib_path):
    from paper_2405_04229_gb300 import binding as B
    d = B.cs_atmosphere_desc()
    d.kind = 7
    h = C.c_void_p()
    assert B.lib().cs_atmosphere_create(C.byref(d), C.byref(h)) == B.CS_ERR_INVALID_ARG
    dd = B.cs_detector_desc()
    dd.n_showers = 0
    assert B.lib().cs_detector_create(C.byref(dd), C.byref(h)) == B.CS_ERR_INVALID_ARG
    out = B.cs_output()
    assert B.lib().cs_propagate(None, 0, None, None, 0, C.byref(out)) == B.CS_ERR_INVALID_ARG
