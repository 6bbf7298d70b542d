"""The C-ABI library builds, loads and exports every entry point declared in
include/biot.h (no GPU needed)."""
import os
import re

from paper_1801_04984_gb300 import binding as B


def test_library_exports_every_declared_symbol():
    from paper_1801_04984_gb300 import build
    build.build()
    lib = B.load()
    names = B.header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_header_has_no_torch_types_and_cites_the_paper():
    txt = open(B.HEADER).read()
    assert not re.search(r"torch|at::|Tensor", txt)
    assert "extern \"C\"" in txt
    for sec in ("Poroelasticity", "Discretisation in Time", "Discretisation in Space", "Monolithic Approach"):
        assert sec in txt


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.dirname(B.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(root, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
