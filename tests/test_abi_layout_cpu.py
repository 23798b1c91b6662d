"""The Python binding's ctypes mirrors of the C-ABI structs agree with the
headers: the C compiler's size and field offsets of every struct, and the
field names in order as the header declares them (a field added on one side
only shifts every later field, or hides in trailing padding).  Host only:
gcc compiles a small program against include/*.h."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2410_06770_gb300 import batch as gb
from paper_2410_06770_gb300 import gett, peaks

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")

# (header, struct name, ctypes mirror)
STRUCTS = [
    ("gett.h", "gett_options", gett.Options),
    ("gett.h", "gett_report", gett.Report),
    ("gett.h", "gett_plan_info", gett.PlanInfo),
    ("gett_batch.h", "gett_problem_desc", gb.ProblemDesc),
    ("gett_batch.h", "gett_batch_options", gb.BatchOptions),
    ("gett_batch.h", "gett_batch_info", gb.BatchInfo),
    ("gett_bench.h", "gett_peaks", peaks._Peaks),
]


def header_fields(header, cname):
    """Field names of `typedef struct cname { ... } cname;`, in order."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(INC, header)).read(), flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    body = re.search(r"typedef struct " + cname + r"\s*\{(.*?)\}\s*" + cname + r"\s*;", text, re.S).group(1)
    names = []
    for decl in body.split(";"):
        decl = re.sub(r"\[[^\]]*\]", "", decl)
        for piece in decl.split(","):
            ids = re.findall(r"[A-Za-z_]\w*", piece)
            if ids:
                names.append(ids[-1])
    return names


@pytest.fixture(scope="module")
def compiled_layout(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>"]
    lines += sorted({f'#include "{h}"' for h, _, _ in STRUCTS})
    lines.append("int main(void) {")
    for _, cname, cls in STRUCTS:
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([gcc, "-I", INC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    return {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}


@pytest.mark.parametrize("header,cname,cls", STRUCTS, ids=[c for _, c, _ in STRUCTS])
def test_mirror_matches_header(compiled_layout, header, cname, cls):
    assert header_fields(header, cname) == [f for f, _ in cls._fields_]
    assert compiled_layout[(cname, "size")] == ctypes.sizeof(cls)
    for fname, _ in cls._fields_:
        assert compiled_layout[(cname, fname)] == getattr(cls, fname).offset, fname
