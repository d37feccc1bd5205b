"""The binding's ctypes structures have the layout of the header's structs: size, and every
member's offset and size, as a C compiler reports them for include/qed.h.  CPU only."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_1311_5551_gb300 import qed

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")

PAIRS = [("qed_table_params", qed.TableParams), ("qed_table_arrays", qed.TableArrays),
         ("qed_allocator", qed.Allocator), ("qed_merge_params", qed.MergeParams), ("qed_soa", qed.Soa),
         ("qed_species_view", qed.SpeciesView), ("qed_field_desc", qed.FieldDesc),
         ("qed_step_params", qed.StepParamsC), ("qed_ledger", qed.Ledger)]


def test_struct_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qed.h"', "int main(void) {"]
    for cname, py in PAIRS:
        lines.append(f'  printf("{cname} . %zu 0\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f'sizeof((({cname}*)0)->{fname}));')
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    c_layout = {(a, b): (int(v), int(w)) for a, b, v, w in (line.split() for line in out.splitlines())}
    py_layout = {}
    for cname, py in PAIRS:
        py_layout[(cname, ".")] = (C.sizeof(py), 0)
        for fname, _ in py._fields_:
            py_layout[(cname, fname)] = (getattr(py, fname).offset, getattr(py, fname).size)
    assert py_layout == c_layout


def test_enum_values_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = {"QED_ELECTRON": qed.ELECTRON, "QED_POSITRON": qed.POSITRON, "QED_PHOTON": qed.PHOTON,
             "QED_FP64": qed.FP64, "QED_MIXED": qed.MIXED, "QED_FIELD_UNIFORM": qed.FIELD_UNIFORM,
             "QED_FIELD_ROTATING_E": qed.FIELD_ROTATING_E, "QED_FIELD_PLANE_LP": qed.FIELD_PLANE_LP,
             "QED_FIELD_PLANE_CP": qed.FIELD_PLANE_CP, "QED_FIELD_GRID": qed.FIELD_GRID}
    lines = ["#include <stdio.h>", '#include "qed.h"', "int main(void) {"]
    lines += [f'  printf("{n} %d\\n", (int){n});' for n in names]
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "enums.c", tmp_path / "enums"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    assert {a: int(b) for a, b in (line.split() for line in out.splitlines())} == names

