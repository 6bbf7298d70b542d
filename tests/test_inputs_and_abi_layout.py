"""Host-side checks without a GPU: the seeded workload generators have the structure the
workloads state (layered fields constant per layer, correlated fields with the stated
standard deviation and correlation, unit-RMS directions, the ragged batch drawn from the
stated sets), and the ctypes structures of the binding match the C declarations field by
field (a mismatch would silently shift every argument behind it)."""
import re

import numpy as np
import pytest

from paper_1801_04984_gb300 import binding as B
from paper_1801_04984_gb300.inputs import batch_instances, correlated_logk_2d, fd_directions, layered_logk


def test_layered_field_is_constant_per_layer():
    n = (8, 6, 16)
    g = layered_logk(n, layer_cells=4, std=1.5, seed=1801).reshape(n[::-1])  # (z, y, x)
    for z0 in range(0, 16, 4):
        blk = g[z0:z0 + 4]
        assert np.all(blk == blk[0, 0, 0])
    layers = g[::4, 0, 0]
    assert len(set(layers.tolist())) == 4
    assert np.array_equal(layered_logk(n, 4, 1.5, 1801), layered_logk(n, 4, 1.5, 1801))


def test_layered_field_std_over_many_layers():
    g = layered_logk((1, 40000), layer_cells=1, std=1.5, seed=3)
    assert abs(g.std() - 1.5) < 0.03


def test_correlated_field_std_and_correlation_length():
    f = correlated_logk_2d(128, std=1.0, corr_cells=8.0, seed=1801)
    assert abs(f.std() - 1.0) < 1e-12 and abs(f.mean()) < 1e-12
    # sample autocorrelation along x and y, averaged over seeds: close to 1 at short lags,
    # decaying over the 8-cell correlation length, small far beyond it
    rho = {}
    for lag in (1, 8, 16, 48):
        vals = []
        for seed in range(6):
            g = correlated_logk_2d(128, std=1.0, corr_cells=8.0, seed=seed).reshape(128, 128)
            vals += [np.mean(g * np.roll(g, lag, axis=1)), np.mean(g * np.roll(g, lag, axis=0))]
        rho[lag] = float(np.mean(vals))
    assert rho[1] > 0.98
    assert 0.6 < rho[8] < 0.92
    assert rho[16] < rho[8] - 0.15
    assert abs(rho[48]) < 0.15


def test_fd_directions_are_unit_rms():
    d = fd_directions(1000, count=20, seed=4984)
    assert d.shape == (20, 1000)
    assert np.allclose(np.sqrt(np.mean(d * d, axis=1)), 1.0)


def test_batch_instances_draw_from_the_stated_sets():
    desc = batch_instances(256, seed=1801)
    assert len(desc) == 256
    assert {d["n"] for d in desc} == {16, 32, 64, 128}
    assert {d["r"] for d in desc} == {0, 1, 2}
    assert [d["seed"] for d in desc] == [1801 + i for i in range(256)]
    assert desc == batch_instances(256, seed=1801)


def _c_struct_fields(name):
    txt = open(B.HEADER).read()
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r";", txt)
    assert m, name
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = re.sub(r"\[.*?\]", "", decl).strip()
        if not decl:
            continue
        # "type a, b" / "const double* const* f": the last identifier of each comma part
        for part in decl.split(","):
            fields.append(re.findall(r"[A-Za-z_][A-Za-z_0-9]*", part)[-1])
    return fields


@pytest.mark.parametrize("cname,ctype", [("biot_mesh", B.Mesh), ("biot_coeffs", B.Coeffs), ("biot_opts", B.Opts),
                                         ("biot_solve_opts", B.SolveOpts), ("biot_stats", B.Stats),
                                         ("biot_batch_item", B.BatchItem)])
def test_binding_structures_match_the_header(cname, ctype):
    c_fields = _c_struct_fields(cname)
    py_fields = [f for f, _ in ctype._fields_]
    # the binding may use a shorter name for a Lame coefficient, nothing else differs
    alias = {"lam": "lambda"}
    assert [alias.get(f, f) for f in py_fields] == c_fields, (cname, c_fields, py_fields)
