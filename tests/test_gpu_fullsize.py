"""Parity at the benchmark's full size: the 256 x 256 P2 Helmholtz workload
(n = 263169, 8445 fronts, depth 13) in the configuration bench.py times
(FP32 fronts, compression four levels above the leaves, eps 1e-6, beta 64)
and with FP64 fronts.

The oracle cannot factor the whole problem in test time, so it checks what it
can compute one node at a time:
* the dense fronts of sampled leaves and of sampled nodes below the switching
  level (each from the oracle's dense elimination of that node's subtree);
* the compressed Schur complement of sampled switching-level nodes, whose
  compression sees the exact S on both sides and the same Philox samples;
* at full size, what every solve must satisfy: GMRES reports convergence and
  the float64 true residual, recomputed on the host, meets the tolerance.
Tolerances as in the small-case parity tests (FP32 fronts ~1e-3 normwise, FP64
to rounding)."""
import numpy as np
import pytest

from ndhss_inputs import helmholtz_impedance
from oracle.frontal import assemble_front, factor_node
from oracle.hss import cluster_tree, hss_compress, hss_dense
from oracle.tree import build_tree
from closeness import rel as _rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EPS, BETA, HL, SEED, LEAF = 1e-6, 64, 4, 0, 64


@pytest.fixture(scope="module")
def nd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_07791_gb300 import build, ndhss
    build.build()
    ndhss.load()
    return ndhss


def workload():
    P = helmholtz_impedance(256, 2, 40.0, seed=0)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, LEAF)
    return P, T


@pytest.fixture(scope="module")
def c2(nd):
    P, T = workload()
    tree = nd.ndhss_build_tree(P.coords, P.A.indptr, P.A.indices, LEAF)
    return dict(P=P, T=T, tree=tree, M=nd.DeviceCSR(P.A))


def _factor(nd, c, prec):
    M = c["M"]
    opts = nd.make_factor_opts(prec=prec, hss_levels=HL, eps_hss=EPS, beta=BETA, k0=32, r=16, seed=SEED)
    return nd.ndhss_factor(c["tree"], M.vtype, M.rowptr, M.col, M.vals, opts)


def dense_refs(T, A, s):
    """(A_ii, L, R, S) of node s by the oracle's dense elimination of its subtree
    (Eq. 3.2 - 3.5); every node below the switching level is dense."""
    S = {k: dense_refs(T, A, k)[3] for k in T.children(s)}
    F = assemble_front(T, s, A, S)
    mi = int(T.node_info[s, 5])
    _, L, R, Sc = factor_node(F, mi)
    return F[:mi, :mi], L, R, Sc


def switching_ref(T, A, s):
    """The oracle's compressed S of a switching-level node: Alg. A.1 on the
    exact S with the parent-conforming cluster tree and the node's stream."""
    Aii, L, R, S = dense_refs(T, A, s)
    mb = int(T.node_info[s, 7])
    p = int(T.node_info[s, 1])
    top = int(np.sum(T.emap_of(s) < T.node_info[p, 5]))
    H = hss_compress(S, cluster_tree(mb, top, BETA), EPS, 32, 16, SEED, stream=2 * s, rank_cap=512)
    return Aii, L, R, hss_dense(H)


def samples(T, seed=0):
    """Sampled leaves, nodes one and two levels below the switching level,
    and switching-level nodes (all with interior and boundary DOFs)."""
    lev, mi, mb = T.f("level"), T.f("m_i"), T.f("m_b")
    Lh = T.depth - HL
    rng = np.random.default_rng(seed)
    ok = (mi > 0) & (mb > 0)
    leaves = np.array([s for s in range(T.nnodes) if ok[s] and not T.children(s)])

    def pick(cand, k):
        return [int(x) for x in rng.choice(cand, size=min(k, cand.size), replace=False)]

    dense = pick(leaves, 6) + pick(np.nonzero(ok & (lev == Lh + 1))[0], 4) + pick(np.nonzero(ok & (lev == Lh + 2))[0], 4)
    switching = pick(np.nonzero(ok & (lev == Lh))[0], 4)
    return dense, switching


def _blocks(nd, f, s, mi, mb):
    return [nd.ndhss_factor_get_block(f, s, w, mi, mb) for w in range(4)]


def _solve_and_check(nd, c, f):
    P, M = c["P"], c["M"]
    b = torch.from_numpy(np.ascontiguousarray(P.b)).cuda()
    x = torch.zeros_like(b)
    st = nd.ndhss_gmres(f, M.rowptr, M.col, M.vals, b, x, tol=1e-8)
    xh = x.cpu().numpy()
    rel = np.linalg.norm(P.A @ xh - P.b) / np.linalg.norm(P.b)
    assert st["converged"] and st["iters"] <= 8, st
    assert rel <= 2e-8, rel


def test_fullsize_mixed_sampled_fronts_and_solve(nd, c2):
    """The benchmark's configuration: FP32 fronts with compression."""
    P, T = c2["P"], c2["T"]
    f = _factor(nd, c2, nd.NDHSS_FP32)
    dense, _ = samples(T)
    assert len(dense) >= 10
    for s in dense:
        mi, mb = int(T.node_info[s, 5]), int(T.node_info[s, 7])
        Aii, L, R, S = dense_refs(T, P.A, s)
        X, Rg, Lg, Sg = _blocks(nd, f, s, mi, mb)
        assert _rel(X, np.linalg.inv(Aii)) <= 2e-2, (s, "Aii^-1", _rel(X, np.linalg.inv(Aii)))
        for name, got, ref in (("R", Rg, R), ("L", Lg, L), ("S", Sg, S)):
            assert _rel(got, ref) <= 2e-3, (s, name, _rel(got, ref))
    _solve_and_check(nd, c2, f)


def test_fullsize_fp64_sampled_fronts_switching_level_and_solve(nd, c2):
    """FP64 fronts: dense blocks to rounding; at the switching level the GPU's
    compressed S against the oracle's Alg. A.1 on the same samples (to
    rounding where both take the same rank decisions, within 50 eps always)."""
    P, T = c2["P"], c2["T"]
    f = _factor(nd, c2, nd.NDHSS_FP64)
    dense, switching = samples(T, seed=1)
    for s in dense:
        mi, mb = int(T.node_info[s, 5]), int(T.node_info[s, 7])
        Aii, L, R, S = dense_refs(T, P.A, s)
        X, Rg, Lg, Sg = _blocks(nd, f, s, mi, mb)
        assert _rel(X, np.linalg.inv(Aii)) <= 1e-8
        for name, got, ref in (("R", Rg, R), ("L", Lg, L), ("S", Sg, S)):
            assert _rel(got, ref) <= 1e-9, (s, name, _rel(got, ref))
    exact = 0
    assert len(switching) == 4
    for s in switching:
        mi, mb = int(T.node_info[s, 5]), int(T.node_info[s, 7])
        Aii, L, R, Sh = switching_ref(T, P.A, s)
        X, Rg, Lg, Sg = _blocks(nd, f, s, mi, mb)
        assert _rel(Rg, R) <= 1e-9 and _rel(Lg, L) <= 1e-9
        e = _rel(Sg, Sh)
        assert e <= 50 * EPS, (s, e)
        exact += e <= 1e-9
    assert exact >= 2
    _solve_and_check(nd, c2, f)


def test_fullsize_mixed_compressed_subtree_matches_oracle(nd, c2):
    """The benchmark's configuration above the switching level: for a seeded
    level-7 node, the oracle factors that node's subtree alone (Alg. 3.4 with
    Alg. A.1 on the same Philox streams, low-rank R strictly above the
    switching level) and every compressed S and low-rank R of the subtree is
    compared with the GPU's FP32 factor of the whole problem.  Both sides
    compress to eps = 1e-6 relative, the GPU from FP32 Schur complements and
    with FP32 sampling (rounding floor ~6e-5 relative on a block's
    estimator), so they agree to the apply-level tolerance of a compressed
    FP32 factor, 1e-3 (normwise and entrywise)."""
    from oracle.hss import factor_compressed
    P, T = c2["P"], c2["T"]
    f = _factor(nd, c2, nd.NDHSS_FP32)
    lev, mi_all, mb_all = T.f("level"), T.f("m_i"), T.f("m_b")
    Lh = T.depth - HL
    rng = np.random.default_rng(7)
    cand = np.nonzero((lev == Lh - 2) & (mi_all > 0) & (mb_all > 0))[0]
    s0 = int(rng.choice(cand))
    fac = factor_compressed(T, P.A, hss_levels=HL, eps=EPS, beta=BETA, k0=32, r=16, seed=SEED, subtree=s0)
    checked_s = checked_r = 0
    worst = 0.0
    for s in range(T.nnodes):
        if fac.S[s] is None or lev[s] > Lh or mb_all[s] == 0:
            continue
        mi, mb = int(mi_all[s]), int(mb_all[s])
        Sg = nd.ndhss_factor_get_block(f, s, 3, mi, mb)
        e = _rel(Sg, fac.S[s])
        worst = max(worst, e)
        assert e <= 1e-3, (s, int(lev[s]), "S", e)
        checked_s += 1
        if lev[s] < Lh and mi > 0:
            Rg = nd.ndhss_factor_get_block(f, s, 1, mi, mb)
            Ro = fac.R[s].matmat(np.eye(mb))
            e = _rel(Rg, Ro)
            worst = max(worst, e)
            assert e <= 1e-3, (s, int(lev[s]), "R", e)
            checked_r += 1
    assert checked_s >= 7 and checked_r >= 3, (checked_s, checked_r)
    print(f"compressed subtree of node {s0}: {checked_s} S and {checked_r} R blocks, worst difference {worst:.2e}")
