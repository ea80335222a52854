"""The C-ABI library loads and exports everything include/bfc.h declares;
argument checks that happen before any CUDA call.  No GPU needed."""
import ctypes
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bfc():
    from paper_1812_00283_gb300 import build
    build.build()
    from paper_1812_00283_gb300 import bfc as b
    return b


def test_exports_every_declared_symbol(bfc):
    names = bfc.header_functions()
    assert "bfc_prepare" in names and "bfc_count_edges" in names
    lib = bfc.library()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_headers_all_checked(bfc):
    inc = os.path.join(ROOT, "include")
    assert sorted(os.listdir(inc)) == ["bfc.h"]


def test_version_and_strings(bfc):
    assert bfc.bfc_version() >= 100
    for code, name in bfc.STATUS.items():
        assert bfc.bfc_status_string(code) == name
    assert bfc.bfc_status_string(99) == "BFC_ERR_UNKNOWN"


def test_options_defaults(bfc):
    o = bfc.bfc_options_init()
    assert (o.validate, o.warp_max_work, o.hash_max_work, o.num_ctas, o.wide_positions,
            o.orientation, o.team_max_work) == (1, 384, 24576, 0, 0, 0, -1)


def test_struct_layouts_match_header(bfc, tmp_path):
    # compile a probe against the public header and compare sizes/offsets with ctypes
    import subprocess
    src = tmp_path / "probe.c"
    src.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "bfc.h"
int main(void) {
  printf("%zu %zu %zu\\n", sizeof(bfc_csr), sizeof(bfc_options), sizeof(bfc_info));
  printf("%zu %zu %zu\\n", offsetof(bfc_csr, adj_u), offsetof(bfc_options, reserved),
         offsetof(bfc_info, max_deg_l));
  printf("%zu %zu %zu\\n", offsetof(bfc_options, team_max_work), offsetof(bfc_info, team_starts),
         sizeof(bfc_server_config));
  printf("%zu %zu\\n", offsetof(bfc_server_config, team_max_work), sizeof(bfc_server_stats));
  printf("%zu %zu\\n", sizeof(bfc_batch_shape), offsetof(bfc_batch_shape, max_layer));
  return 0;
}
''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes[:3] == [ctypes.sizeof(bfc.bfc_csr), ctypes.sizeof(bfc.bfc_options),
                         ctypes.sizeof(bfc.bfc_info)]
    assert sizes[3:6] == [bfc.bfc_csr.adj_u.offset, bfc.bfc_options.reserved.offset,
                          bfc.bfc_info.max_deg_l.offset]
    assert sizes[6:11] == [bfc.bfc_options.team_max_work.offset, bfc.bfc_info.team_starts.offset,
                           ctypes.sizeof(bfc.bfc_server_config), bfc.bfc_server_config.team_max_work.offset,
                           ctypes.sizeof(bfc.bfc_server_stats)]
    assert sizes[11:] == [ctypes.sizeof(bfc.bfc_batch_shape), bfc.bfc_batch_shape.max_layer.offset]


@pytest.mark.parametrize("case", ["null", "negative", "too_many_edges", "bad_option", "null_ptr"])
def test_argument_errors_before_cuda(bfc, case):
    lib = bfc.library()
    h = ctypes.c_void_p()
    opts = bfc.bfc_options_init()
    if case == "null":
        rc = lib.bfc_prepare(None, None, None, ctypes.byref(h))
    else:
        csr = bfc.bfc_csr(3, 3, 4, 1234, 5678)
        if case == "negative":
            csr.num_u = -1
        elif case == "too_many_edges":
            csr.num_edges = 1 << 31
        elif case == "bad_option":
            opts.warp_max_work = 100000
        elif case == "null_ptr":
            csr.off_u = None
        rc = lib.bfc_prepare(ctypes.byref(csr), ctypes.byref(opts), None, ctypes.byref(h))
    assert rc == 1
    assert bfc.bfc_last_error()


def test_null_graph_calls(bfc):
    lib = bfc.library()
    assert lib.bfc_count(None, None, None) == 1
    assert lib.bfc_sync(None, None) == 1
    lib.bfc_release(None)


@pytest.mark.parametrize("case", ["max_layer", "graphs", "orientation", "team", "reserved"])
def test_batch_plan_argument_errors_before_cuda(bfc, case):
    # shape and option checks come before any device work
    lib = bfc.library()
    h = ctypes.c_void_p()
    shape = bfc.bfc_batch_shape(100, 100, 500, 4, 50)
    opts = bfc.bfc_options_init()
    if case == "max_layer":
        shape.max_layer = 65536
    elif case == "graphs":
        shape.num_graphs = 0
    elif case == "orientation":
        opts.orientation = 1
    elif case == "team":
        opts.team_max_work = 4096
    else:
        shape.reserved[2] = 1
    rc = lib.bfc_batch_plan_create(ctypes.byref(shape), ctypes.byref(opts), None, ctypes.byref(h))
    assert rc == 1 and h.value is None
    assert bfc.bfc_last_error()
