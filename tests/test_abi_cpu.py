"""C ABI checks that need no GPU: symbols, host validation, host AMG setup
against the oracle (aggregates bit-exact), dt bound against the oracle."""
import os
import re

import numpy as np
import pytest

import eqs_inputs as ei
from oracle import amg, dtbound, system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def E():
    from paper_1612_09447_gb300 import build, eqs

    if not os.path.exists(build.LIB):
        build.build()
    eqs.lib()
    return eqs


def test_exports_every_header_symbol(E):
    hdr = open(os.path.join(ROOT, "include", "eqs.h")).read()
    names = set(re.findall(r"\b(eqs_[A-Za-z_0-9]+)\s*\(", hdr))
    assert len(names) >= 17
    L = E.lib()
    for n in sorted(names):
        assert hasattr(L, n), n


def test_mesh_validation(E):
    p = ei.make_problem(3)
    bad = p.tets.copy()
    bad[5, [2, 3]] = bad[5, [3, 2]]
    with pytest.raises(E.EqsError) as ex:
        E.eqs_mesh_create(p.xyz, bad, p.node_tag)
    assert ex.value.status == E.EQS_ERR_MESH
    oob = p.tets.copy()
    oob[0, 0] = p.n_nodes
    with pytest.raises(E.EqsError) as ex:
        E.eqs_mesh_create(p.xyz, oob, p.node_tag)
    assert ex.value.status == E.EQS_ERR_MESH
    tag = p.node_tag.copy()
    tag[0] = 3
    with pytest.raises(E.EqsError):
        E.eqs_mesh_create(p.xyz, p.tets, tag)
    xyz = p.xyz.copy()
    xyz[3, 1] = np.nan
    with pytest.raises(E.EqsError):
        E.eqs_mesh_create(xyz, p.tets, p.node_tag)
    with pytest.raises(E.EqsError):
        E.eqs_mesh_create(p.xyz, p.tets, np.ones(p.n_nodes, np.uint8))  # no free node
    ctx = E.eqs_mesh_create(p.xyz, p.tets, p.node_tag)
    with pytest.raises(E.EqsError) as ex:  # setup before materials
        E.eqs_amg_setup(ctx)
    assert ex.value.status == E.EQS_ERR_STATE
    with pytest.raises(E.EqsError):
        E.eqs_set_materials(ctx, np.full(p.n_tets, 2, np.uint8), p.materials)
    E.eqs_destroy(ctx)


def test_dt_bound_matches_oracle(E):
    p = ei.make_problem(2)
    ctx = E.eqs_mesh_create(p.xyz, p.tets, p.node_tag)
    E.eqs_set_materials(ctx, p.tet_mat, p.materials)
    for s in (2, 10, 20, 64):
        assert E.eqs_rkc_dt_bound(ctx, s) == pytest.approx(dtbound.dt_bound(p.materials, s), rel=1e-12)
    assert E.eqs_rkc_dt_bound(ctx, 1) < 0
    E.eqs_destroy(ctx)


def _host_setup(E, p):
    ctx = E.eqs_mesh_create(p.xyz, p.tets, p.node_tag)
    E.eqs_set_materials(ctx, p.tet_mat, p.materials)
    try:
        E.eqs_amg_setup(ctx)
    except E.EqsError as e:  # no GPU here: the host hierarchy is still built
        assert e.status == E.EQS_ERR_CUDA
    return ctx


@pytest.mark.parametrize("cfg,N", [(0, 12), (2, 10), (4, 16), (1, 20)])
def test_host_amg_matches_oracle(E, cfg, N):
    p = ei.config_problem(cfg, N=N)
    ctx = _host_setup(E, p)
    rows, nnz = E.eqs_amg_info(ctx)
    H = amg.SAHierarchy(system.EQSSystem(p).Mff)
    assert rows == [l.n for l in H.levels]
    for l in range(len(rows) - 1):
        agg = E.eqs_amg_aggregates(ctx, l, rows[l])
        assert np.array_equal(agg, H.levels[l].agg)
    assert nnz[0] == H.levels[0].A.nnz
    E.eqs_destroy(ctx)


@pytest.mark.parametrize("N,jitter", [(4, 0.0), (5, 0.2)])
def test_host_amg_matches_oracle_p2(E, N, jitter):
    """Quadratic tets: the host assembly of M (10-node shape functions,
    4-point rule) gives the oracle's matrix pattern and the same hierarchy."""
    p = ei.make_problem_p2(N, jitter=jitter, seed=3)
    ctx = _host_setup(E, p)
    rows, nnz = E.eqs_amg_info(ctx)
    H = amg.SAHierarchy(system.EQSSystem(p).Mff)
    assert rows == [l.n for l in H.levels]
    assert nnz[0] == H.levels[0].A.nnz
    for l in range(len(rows) - 1):
        assert np.array_equal(E.eqs_amg_aggregates(ctx, l, rows[l]), H.levels[l].agg)
    E.eqs_destroy(ctx)


def test_p2_mesh_validation(E):
    p = ei.make_problem_p2(2)
    bad = p.tets.copy()
    bad[0, 7] = p.n_nodes  # a midpoint index out of range
    with pytest.raises(E.EqsError) as ex:
        E.eqs_mesh_create(p.xyz, bad, p.node_tag)
    assert ex.value.status == E.EQS_ERR_MESH


@pytest.mark.parametrize("field,value", [("pod_k", 0), ("pod_k", 17), ("pod_m", 0), ("pod_m", 13),
                                         ("pod_min_iters", -1), ("spe_n", 7), ("cheb_degree", 5),
                                         ("rtol", 0.0), ("precision", 2), ("coarse_split", 2),
                                         ("defer_sums", 4), ("defer_sums", -1)])
def test_invalid_options_are_rejected_before_any_device_work(E, field, value):
    p = ei.make_problem(2)
    ctx = E.eqs_mesh_create(p.xyz, p.tets, p.node_tag)
    E.eqs_set_materials(ctx, p.tet_mat, p.materials)
    o = E.eqs_opts_default()
    setattr(o, field, value)
    with pytest.raises(E.EqsError) as ex:
        E.eqs_amg_setup(ctx, o)
    assert ex.value.status == E.EQS_ERR_ARG
    E.eqs_destroy(ctx)


def test_call_order_errors(E):
    p = ei.make_problem(2)
    ctx = E.eqs_mesh_create(p.xyz, p.tets, p.node_tag)
    for call in (lambda: E.eqs_apply_K(ctx, None, None), lambda: E.eqs_get_step_stats(ctx)):
        with pytest.raises(E.EqsError) as ex:
            call()
        assert ex.value.status == E.EQS_ERR_STATE
    E.eqs_destroy(ctx)


def test_option_defaults_match_the_header(E):
    """eqs_opts_default fills the values include/eqs.h documents."""
    o = E.eqs_opts_default()
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "eqs.h")).read()
    doc = hdr[hdr.index("/* Fill *o with the defaults"):]
    doc = " ".join(doc[:doc.index("*/")].replace("*", " ").split())
    for field in ("split_m", "pod_k", "pod_m", "pod_min_iters", "fill_lanes", "coarse_split", "defer_sums",
                  "spe_n", "max_iter", "persistent", "host_loop"):
        m = re.search(rf"\b{field} (\d+)", doc)
        assert m, field
        assert getattr(o, field) == int(m.group(1)), field
    assert o.precision == E.EQS_PREC_FP64 and o.rtol == 1e-8 and o.flexible == 1


def test_solver_rejects_unknown_options():
    """A misspelt solver option raises before anything is created (ctypes
    would otherwise store it as a plain attribute and ignore it)."""
    from paper_1612_09447_gb300 import eqs

    with pytest.raises(TypeError, match="cheb_degre"):
        eqs.Solver(ei.make_problem(2), cheb_degre=1)
