"""The C-ABI library builds, loads, and exports every function include/*.h declares (CPU only:
no compute call is made)."""
import ctypes as C
import glob
import os
import re

from paper_2511_22852_gb300 import binding as Bd
from paper_2511_22852_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sph_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["sph_set_eos_table", "sph_init_event", "sph_step", "sph_read_fields", "sph_free_event",
                 "sph_free_eos", "sph_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    path = build_lib.build()
    lib = C.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(Bd.EXPORTS) <= declared_functions()


def test_struct_sizes_match_the_header_layout():
    # the ctypes mirrors follow the C layout (natural alignment, 64-bit pointers)
    assert C.sizeof(Bd.EosDesc) == 8 * 7 + 4 * 6 + 8 * 8 + 8 * 5 + 8
    assert C.sizeof(Bd.EventDesc) == 4 * 4 + 8 * 4 + 8 * 6 + 8 * 7 + 4 * 2 + 8 + 4 * 2 + 8 + 8 * 3
    assert C.sizeof(Bd.FieldBufs) == 8 * 18 + 8 + 8
    assert C.sizeof(Bd.Totals) == 8 * 7 + 4 * 2 + 8 * 7
    assert C.sizeof(Bd.ServerDesc) == 4 * 2 + 8 * 4 + 4 * 2 + 8
    assert C.sizeof(Bd.ServerStats) == 8 * 8 + 4 * 2 + 8 + 8 + 8
