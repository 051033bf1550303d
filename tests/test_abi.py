"""The C-ABI library builds, loads and exports every entry point of include/bfs.h (CPU only; no compute)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bfs.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\**\s*(bfs_[a-z0-9_]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_1705_04590_gb300 as bfs
    bfs.build()
    return ctypes.CDLL(bfs.LIB)


def test_header_parses():
    names = declared_functions()
    for must in ["bfs_graph_create_from_edges", "bfs_graph_create_from_csr", "bfs_graph_info", "bfs_graph_destroy",
                 "bfs_run", "bfs_run_multi", "bfs_server_create", "bfs_server_add_graph", "bfs_submit",
                 "bfs_poll", "bfs_wait", "bfs_server_destroy", "bfs_status_string", "bfs_last_error"]:
        assert must in names, must


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_1705_04590_gb300 as bfs
    bound = {name for name, _, _ in bfs.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_status_strings_without_gpu(lib):
    lib.bfs_status_string.restype = ctypes.c_char_p
    lib.bfs_version.restype = ctypes.c_char_p
    assert lib.bfs_status_string(0) == b"BFS_OK"
    assert lib.bfs_status_string(4) == b"BFS_ERR_TIMEOUT"
    assert b"sm_103a" in lib.bfs_version()


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors have the sizes and offsets the C compiler gives the header's structs."""
    import subprocess
    import paper_1705_04590_gb300._lib as L
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "bfs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(bfs_options), sizeof(bfs_level_record),
         sizeof(bfs_stats), sizeof(bfs_allocator), sizeof(bfs_dcsc_layout), offsetof(bfs_options, timeout_ms),
         offsetof(bfs_options, ctas_per_sm), offsetof(bfs_options, cluster_size), offsetof(bfs_stats, vertices_reached));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(L.Options), ctypes.sizeof(L.LevelRecord), ctypes.sizeof(L.Stats),
            ctypes.sizeof(L.Allocator), ctypes.sizeof(L.DcscLayout), L.Options.timeout_ms.offset,
            L.Options.ctas_per_sm.offset, L.Options.cluster_size.offset, L.Stats.vertices_reached.offset]
    assert got == want
