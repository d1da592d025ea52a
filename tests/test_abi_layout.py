"""The ctypes binding mirrors include/pt.h: every struct's size and every
field's offset, and the status codes, flags and limits, as a C compiler lays
them out from the header itself.  A field added, reordered or retyped on one
side only fails here, on the CPU, before any call reaches a kernel.  The
oracle's own binding is checked against oracle/oracle.h the same way."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2008_13461_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "pt_layer": L.Layer, "pt_geometry": L.Geometry, "pt_pair_cuts": L.PairCuts, "pt_ca_cuts": L.CaCuts,
    "pt_cuts": L.Cuts, "pt_fit_params": L.FitParams, "pt_tuning": L.Tuning, "pt_capacity": L.Capacity,
    "pt_config": L.Config, "pt_hits": L.Hits, "pt_cells": L.Cells, "pt_edges": L.Edges, "pt_tuples": L.Tuples,
    "pt_tracks": L.Tracks, "pt_counts": L.Counts, "pt_vertex_tracks": L.VertexTracks,
    "pt_vertex_cuts": L.VertexCuts, "pt_vertices": L.Vertices, "pt_kernel_time": L.KernelTime,
}

CONSTANTS = {
    "PT_N_LAYERS": L.N_LAYERS, "PT_MAX_PAIRS": L.MAX_PAIRS, "PT_NMAX": L.NMAX,
    "PT_OK": L.PT_OK, "PT_ERR_INVALID_ARG": L.PT_ERR_INVALID_ARG, "PT_ERR_CAPACITY": L.PT_ERR_CAPACITY,
    "PT_ERR_INPUT": L.PT_ERR_INPUT, "PT_ERR_CUDA": L.PT_ERR_CUDA, "PT_ERR_TOO_LARGE": L.PT_ERR_TOO_LARGE,
    "PT_FLAG_CELLS": L.FLAG_CELLS, "PT_FLAG_EDGES": L.FLAG_EDGES, "PT_FLAG_TUPLES": L.FLAG_TUPLES,
    "PT_FLAG_TRACKS": L.FLAG_TRACKS, "PT_FLAG_INPUT": L.FLAG_INPUT,
    "PT_VTX_MAX_TRACKS": L.PT_VTX_MAX_TRACKS, "PT_VTX_MAX_VERTICES": L.PT_VTX_MAX_VERTICES,
    "PT_VTX_EVENT_TOO_LARGE": L.PT_VTX_EVENT_TOO_LARGE, "PT_VTX_TOO_MANY": L.PT_VTX_TOO_MANY,
    "PT_VTX_INTERNAL": L.PT_VTX_INTERNAL,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    """sizeof / offsetof / constant values printed by a C program built
    against the header."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pt.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'printf("size {cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("off {cname} {f} %zu\\n", offsetof({cname}, {f}));')
    for name in CONSTANTS:
        lines.append(f'printf("const {name} %lld\\n", (long long)({name}));')
    lines += ["return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        kind, *key, val = ln.split()
        got[(kind, *key)] = int(val)
    return got


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_struct_matches_the_header(c_layout, cname):
    cls = STRUCTS[cname]
    assert C.sizeof(cls) == c_layout[("size", cname)], cname
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == c_layout[("off", cname, f)], f"{cname}.{f}"


def test_constants_match_the_header(c_layout):
    for name, v in CONSTANTS.items():
        assert v == c_layout[("const", name)], name


def test_oracle_binding_matches_its_header(tmp_path):
    """The same check for the oracle's ctypes mirror of oracle/oracle.h (a
    drifted field there would feed the oracle wrong cuts or read its results
    from the wrong offsets)."""
    import oracle
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"or_pair": oracle._Pair, "or_region": oracle._Region, "or_cuts": oracle._Cuts,
               "or_fitpar": oracle._FitPar, "or_input": oracle._Input, "or_tuple": oracle._Tuple,
               "or_result": oracle._Result}
    lines = ["#include <stdio.h>", "#include <stddef.h>", "#include <stdint.h>", '#include "oracle.h"',
             "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("size {cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("off {cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src, exe = tmp_path / "olayout.c", tmp_path / "olayout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "oracle"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        kind, *key, val = ln.split()
        got[(kind, *key)] = int(val)
    for cname, cls in structs.items():
        assert C.sizeof(cls) == got[("size", cname)], cname
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == got[("off", cname, f)], f"{cname}.{f}"
