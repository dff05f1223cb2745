"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every declared symbol, and its tree builder matches the oracle bit for bit."""
import os
import re

import numpy as np
import pytest

from ndhss_inputs import helmholtz_impedance, poisson_dirichlet
from oracle.tree import build_tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nd():
    from paper_2105_07791_gb300 import build, ndhss
    build.build()
    ndhss.load()
    return ndhss


def test_exports_every_declared_symbol(nd):
    hdr = open(os.path.join(ROOT, "include", "ndhss.h")).read()
    declared = set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(ndhss_\w+)\s*\(", hdr, flags=re.M))
    assert len(declared) >= 12
    lib = nd.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(nd.EXPORTED)
    assert nd.ndhss_version().startswith("ndhss")


TREE_KEYS = ("perm", "node_info", "blist", "emap", "e_off", "e_row", "e_col", "e_idx")


@pytest.mark.parametrize("case", ["c1", "p1_odd", "p2_small", "helm_p1", "leaf16", "tiny", "single_leaf", "elastic_dg"])
def test_tree_bit_exact_vs_oracle(nd, case):
    leaf = 64
    if case == "c1":
        P = poisson_dirichlet(64)
    elif case == "p1_odd":
        P = poisson_dirichlet(37, seed=3)
    elif case == "p2_small":
        P = helmholtz_impedance(24, 2, 12.0)
    elif case == "helm_p1":
        P = helmholtz_impedance(45, 1, 9.0)
    elif case == "leaf16":
        P, leaf = helmholtz_impedance(20, 1, 4.0), 16
    elif case == "elastic_dg":
        from ndhss_inputs.elastic import elastic_sipg
        P, leaf = elastic_sipg(14, seed=1), 60          # 12 DOFs per cell share its coordinate
    elif case == "tiny":
        P, leaf = poisson_dirichlet(4), 2
    else:
        P = poisson_dirichlet(6)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, leaf)
    e = nd.ndhss_tree_export(nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, leaf))
    for k in TREE_KEYS:
        assert np.array_equal(e[k], getattr(T, k)), k


def test_tree_bit_exact_full_c2(nd):
    """The benchmark workload (P2, 256 x 256 cells, n = 263169): identical tree."""
    P = helmholtz_impedance(256, 2, 40.0)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    e = nd.ndhss_tree_export(nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 64))
    assert T.nnodes == 8445 and T.depth == 13 and T.node_info[-1, 5] == 1539
    for k in TREE_KEYS:
        assert np.array_equal(e[k], getattr(T, k)), k


def test_tree_with_gaps_and_empty_boxes(nd):
    """DOFs on a lattice with holes: empty boxes become size-0 leaves in both builders."""
    P = poisson_dirichlet(32)
    keep = np.nonzero((P.coords[:, 0] < 10) | (P.coords[:, 0] > 20) | (P.coords[:, 1] < 12))[0]
    A = P.A[keep][:, keep].tocsr()
    A.sort_indices()
    coords = P.coords[keep]
    T = build_tree(coords, A.indptr, A.indices, 20)
    e = nd.ndhss_tree_export(nd.ndhss_build_tree(coords, A.indptr, A.indices, 20))
    for k in TREE_KEYS:
        assert np.array_equal(e[k], getattr(T, k)), k
    assert np.any(T.f("m_i") + T.f("m_b") == 0)


def test_invalid_arguments_return_error_codes(nd):
    P = poisson_dirichlet(8)
    bad = P.A.indices.copy()
    bad[3] = 10 ** 6
    with pytest.raises(nd.NdhssError) as ei:
        nd.ndhss_build_tree(P.coords, P.A.indptr, bad, 16)
    assert ei.value.code == 1 and "out of range" in str(ei.value)
    with pytest.raises(nd.NdhssError):
        nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, 0)


def test_batched_tree_is_the_forest_of_the_oracle_trees(nd):
    """ndhss_build_tree_batched: every problem's oracle tree, node ids, DOF
    positions, B lists and entry indices shifted by the problems before it,
    roots on level 0 (the block-diagonal matrix of the batch)."""
    probs = [poisson_dirichlet(9), helmholtz_impedance(13, 1, 5.0), poisson_dirichlet(20, seed=2),
             helmholtz_impedance(6, 2, 3.0)]
    leaf = 16
    e = nd.ndhss_tree_export(
        nd.ndhss_build_tree_batched([(P.coords, P.A.indptr, P.A.indices) for P in probs], leaf))
    want = {k: [] for k in TREE_KEYS}
    dof = node = boff = eoff = 0
    want["e_off"] = [np.zeros(1, np.int32)]
    for P in probs:
        T = build_tree(P.coords, P.A.indptr, P.A.indices, leaf)
        ni = T.node_info.copy()
        for f in (1, 2, 3):
            ni[:, f] = np.where(ni[:, f] >= 0, ni[:, f] + node, ni[:, f])
        ni[:, 4] += dof
        ni[:, 6] += boff
        want["node_info"].append(ni)
        want["perm"].append(T.perm + dof)
        want["blist"].append(T.blist + dof)
        want["emap"].append(T.emap)
        want["e_off"].append(T.e_off[1:] + eoff)
        want["e_row"].append(T.e_row)
        want["e_col"].append(T.e_col)
        want["e_idx"].append(T.e_idx + eoff)
        dof += P.A.shape[0]
        node += ni.shape[0]
        boff += T.blist.size
        eoff += P.A.nnz
    for k in TREE_KEYS:
        assert np.array_equal(e[k], np.concatenate(want[k])), k
    roots = e["node_info"][e["node_info"][:, 1] < 0]
    assert roots.shape[0] == len(probs) and np.all(roots[:, 0] == 0)
    # the batch's CSR layout
    A, off = nd.batch_csr([P.A for P in probs])
    assert off[-1] == A.shape[0] == dof and A.nnz == eoff


def test_batched_tree_rejects_a_bad_problem(nd):
    P = poisson_dirichlet(8)
    bad_col = P.A.indices.copy()
    bad_col[3] = P.A.shape[0] + 5
    with pytest.raises(nd.NdhssError, match="problem 1"):
        nd.ndhss_build_tree_batched([(P.coords, P.A.indptr, P.A.indices), (P.coords, P.A.indptr, bad_col)], 16)


def test_binding_structs_and_constants_match_the_header(nd, tmp_path):
    """The ctypes mirrors of the header's structs have the C layout (size and
    every field's offset, as gcc lays them out), and the binding's status,
    value-type and precision constants equal the header's enumerators."""
    import ctypes
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"ndhss_factor_opts": nd.FactorOpts, "ndhss_gmres_opts": nd.GmresOpts,
               "ndhss_gmres_stats": nd.GmresStats, "ndhss_factor_stats": nd.FactorStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ndhss.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    enums = ["NDHSS_OK", "NDHSS_ERR_INVALID_ARG", "NDHSS_ERR_OOM", "NDHSS_ERR_SINGULAR", "NDHSS_ERR_RANK_CAP",
             "NDHSS_ERR_NOT_CONVERGED", "NDHSS_ERR_TIMEOUT", "NDHSS_ERR_CUDA", "NDHSS_ERR_INTERNAL", "NDHSS_R64",
             "NDHSS_C128", "NDHSS_FP64", "NDHSS_FP32", "NDHSS_FP32_TF32", "NDHSS_FP32_BF16"]
    for e in enums:
        lines.append(f'printf("enum {e} %d\\n", (int){e});')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, v = line.split()
            got[(a, b)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
    status = {v: k for k, v in nd.STATUS.items()}
    for e in enums[:9]:
        name = e.replace("NDHSS_ERR_", "").replace("NDHSS_", "")
        assert got[("enum", e)] == status[name], e
    for e in enums[9:]:
        assert got[("enum", e)] == getattr(nd, e), e
