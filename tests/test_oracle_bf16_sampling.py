"""Why the HSS sampling stays FP32: Alg. A.1 (oracle) with its sampling
product formed from BF16-rounded operands, on a Schur complement of a
Helmholtz front (exact entries, exact accumulation).  BF16 estimator samples
never certify eps = 1e-6 (the estimate sits on the BF16 rounding floor), so
sampling runs to the matrix size and no compression is left; BF16 samples
with a full-precision estimator meet eps but with several times the rank."""
import numpy as np

import oracle.hss as H
from ndhss_inputs import helmholtz_impedance
from oracle.frontal import assemble_front, factor_node
from oracle.tree import build_tree


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return bf16(x.real) + 1j * bf16(x.imag)
    u = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


class Bf16Op:
    """S through products from BF16-rounded S and X (all of them, or only
    blocks wider than ``exact_below`` columns), and exact entries."""

    def __init__(self, S, exact_below=0):
        self.S, self.Sb, self.shape, self.dtype, self.cut = S, bf16(S), S.shape, S.dtype, exact_below

    def matmat(self, X):
        return self.Sb @ bf16(X) if X.shape[1] > self.cut else self.S @ X

    def entries(self, I, J):
        return self.S[np.ix_(I, J)]


def _largest_schur():
    P = helmholtz_impedance(40, 2, 16.0, seed=0)
    T = build_tree(P.coords, P.A.indptr, P.A.indices, 64)
    keep, best = {}, None
    for s in range(T.nnodes):
        F = assemble_front(T, s, P.A, keep)
        S = factor_node(F, int(T.node_info[s, 5]))[3]
        for k in T.children(s):
            keep.pop(k, None)
        keep[s] = S
        p = int(T.node_info[s, 1])
        if p >= 0 and (best is None or S.shape[0] > best[1].shape[0]):
            best = (s, S, int(np.sum(T.emap_of(s) < T.node_info[p, 5])))
    return best


def test_bf16_sampling_loses_the_compression():
    s, S, top = _largest_schur()
    n = S.shape[0]
    assert n >= 150
    tree = H.cluster_tree(n, top, 64)
    eps = 1e-6
    ref = np.linalg.norm(S)
    full = H.hss_compress(S, tree, eps, seed=1, stream=2 * s)
    assert np.linalg.norm(H.hss_dense(full) - S) <= 10 * eps * ref
    # BF16 estimator samples: eps is never certified, sampling runs to the size of the matrix
    allb = H.hss_compress(Bf16Op(S), tree, eps, seed=1, stream=2 * s)
    assert allb.samples >= n - 16 and allb.kmax() >= 4 * full.kmax(), (allb.samples, allb.kmax(), full.kmax())
    # BF16 samples, full-precision estimator: eps met, with several times the rank
    mixed = H.hss_compress(Bf16Op(S, exact_below=16), tree, eps, seed=1, stream=2 * s)
    assert np.linalg.norm(H.hss_dense(mixed) - S) <= 10 * eps * ref
    assert mixed.kmax() >= 2 * full.kmax(), (mixed.kmax(), full.kmax())
