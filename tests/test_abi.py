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


def test_library_time_tables_match_the_oracle():
    """The CUDA path's host-side dG(r) tables (Radau nodes and weights, D, and the real block
    form of the time operator used by the preconditioner) agree with the oracle's exact
    change of basis from the Legendre matrices, and V Lambda V^{-1} reproduces M_t^{-1} D."""
    import numpy as np
    from oracle import timebasis as tb
    for r in (0, 1, 2):
        t = B.time_tables(r)
        Mt, D = tb.radau_matrices(r)
        assert np.allclose(t["nodes"], tb.radau_right_nodes(r), atol=1e-15)
        assert np.allclose(t["w"], np.diag(Mt), atol=1e-14) and np.allclose(Mt, np.diag(np.diag(Mt)), atol=1e-13)
        assert np.allclose(t["D"], D, atol=1e-12)
        assert np.allclose(t["phi0"], tb.basis_values(np.array([0.0]), r, "radau")[:, 0], atol=1e-13)
        Lam = np.diag(t["lam"])
        p = t["pair"]
        if p >= 0:
            Lam[p, p + 1], Lam[p + 1, p] = t["pair_beta"], -t["pair_beta"]
        T = np.linalg.solve(Mt, D)
        assert np.allclose(t["V"] @ Lam @ np.linalg.inv(t["V"]), T, atol=1e-11), r
        assert np.allclose(t["W"], np.linalg.inv(t["V"]) @ np.linalg.inv(Mt), atol=1e-10)
        assert (p >= 0) == (r >= 1)  # dG(1) and dG(2) have one complex pair


def test_binding_constants_equal_the_header_enums():
    """Every BIOT_<NAME> = value enumerator of include/biot.h has the same value as the
    binding's <NAME> constant (the binding passes these integers through the C ABI)."""
    txt = open(B.HEADER).read()
    enums = {}
    for block in re.finditer(r"\benum\s*\{([^}]*)\}", txt):
        body = re.sub(r"/\*.*?\*/", "", block.group(1), flags=re.S)
        enums.update({m.group(1): int(m.group(2)) for m in re.finditer(r"\bBIOT_([A-Z0-9_]+)\s*=\s*(-?\d+)", body)})
    assert len(enums) >= 25
    for name, value in enums.items():
        assert hasattr(B, name), name
        assert getattr(B, name) == value, (name, getattr(B, name), value)
