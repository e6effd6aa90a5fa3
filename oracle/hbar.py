"""Closed-form spin-free dressed Hamiltonian H-bar (<= two-body) for a closed-shell reference.

Passage followed: the downfolded Hamiltonian of Eqs. (5)-(8) with N = 1, in the SES-CC
reading of the flow's sigma: every active space of a sweep sees the same similarity-
transformed Hamiltonian H-bar = e^{-T} H e^{T} built from the current global amplitude pool
T = T1 + T2, normal ordered with respect to the reference Phi and truncated to one- and
two-body terms ("dressed one- and two-body integrals").

Conventions.  Orbitals 0..nocc-1 are occupied (i, j, k, l, m, n), nocc..n-1 virtual
(a, b, c, d, e, f; stored with local index a - nocc).  t1[i, a] = t_i^a and
t2[i, j, a, b] = t_ij^ab (alpha-beta amplitude, t2[i,j,a,b] = t2[j,i,b,a]).  The result is
    H-bar_<=2 = E0 + sum_pq F[p,q] {E_pq} + 1/2 sum_pqrs W[p,q,r,s] {E_pq E_rs},
{.} = normal order with respect to Phi; W[p,q,r,s] has creators p, r and annihilators q, s
and the pair symmetry W[p,q,r,s] = W[r,s,p,q].

Construction.  T1 enters exactly through the orbital similarity transformation
e^{-T1} H e^{T1} (creators transformed by 1 - K, annihilators by 1 + K, K_ai = t_i^a, K^2 = 0).
T2 is then added through its connected contractions: one- and two-body parts of
[H~, T2] and the fully contracted quadratic term of 1/2 [[H~, T2], T2] (the latter only
reaches the doubly excited block).  The spin-free expressions below were obtained by
spin-integrating the spin-orbital contractions; they are pinned, block by block, against
``oracle.hbar_brute`` (exact Fock-space extraction), and the residual blocks against
determinant-space e^{-T} H e^{T} Phi at ten orbitals.
"""
from __future__ import annotations

import numpy as np

ein = lambda spec, *ops: np.einsum(spec, *ops, optimize=True)  # noqa: E731


def t1_transform(h: np.ndarray, g: np.ndarray, t1: np.ndarray, nocc: int):
    """h~ = (1-K) h (1+K); g~_pqrs = sum X_pp' Y_q'q X_rr' Y_s's g_p'q'r's' (X = 1-K, Y = 1+K)."""
    n = h.shape[0]
    K = np.zeros((n, n))
    K[nocc:, :nocc] = t1.T
    X = np.eye(n) - K
    Y = np.eye(n) + K
    ht = X @ h @ Y
    gt = ein("pP,Qq,rR,Ss,PQRS->pqrs", X, Y, X, Y, g)
    return ht, gt


def reference_terms(ht: np.ndarray, gt: np.ndarray, nocc: int):
    """E~ = <Phi|H~|Phi> and the normal-ordered one-body part f~ of H~."""
    o = slice(0, nocc)
    e = 2.0 * np.trace(ht[o, o]) + 2.0 * ein("kkll->", gt[o, o, o, o]) - ein("kllk->", gt[o, o, o, o])
    f = ht + 2.0 * ein("pqkk->pq", gt[:, :, o, o]) - ein("pkkq->pq", gt[:, o, o, :])
    return e, f


def _blocks(gt, nocc):
    o, v = slice(0, nocc), slice(nocc, gt.shape[0])
    return o, v


def fock_oo_vv(f, gt, t2, nocc):
    """F[m,i] (oo) and F[a,e] (vv) blocks of H-bar."""
    o, v = _blocks(gt, nocc)
    u = 2.0 * t2 - t2.transpose(0, 1, 3, 2)
    g_ovov = gt[o, v, o, v]
    foo = f[o, o] + ein("menf,inef->mi", g_ovov, u)
    fvv = f[v, v] - ein("menf,mnaf->ae", g_ovov, u)
    return foo, fvv


def energy(ht, gt, t2, nocc):
    """E0 = <Phi|H-bar|Phi> (the CCSD energy functional for the pool)."""
    o, v = _blocks(gt, nocc)
    e_ref, _ = reference_terms(ht, gt, nocc)
    u = 2.0 * t2 - t2.transpose(0, 1, 3, 2)
    return e_ref + ein("iajb,ijab->", gt[o, v, o, v], u)


def singles_residual(f, gt, t2, nocc):
    """F[a,i] (vo block) = <Phi_i^a|H-bar|Phi>."""
    o, v = _blocks(gt, nocc)
    u = 2.0 * t2 - t2.transpose(0, 1, 3, 2)
    r = f[v, o].copy()
    r += ein("me,imae->ai", f[o, v], u)
    r += ein("aemf,imef->ai", gt[v, v, o, v], u)
    r -= ein("mine,mnae->ai", gt[o, o, o, v], u)
    return r


def oooo_block(gt, t2, nocc):
    o, v = _blocks(gt, nocc)
    return gt[o, o, o, o] + ein("kelf,ijef->kilj", gt[o, v, o, v], t2)


def doubles_residual(f, gt, t2, nocc, foo=None, fvv=None, woooo=None):
    """W[a,i,b,j] (vovo block) = <Phi_{i alpha j beta}^{a alpha b beta}|H-bar|Phi>, returned as R[i,j,a,b]."""
    o, v = _blocks(gt, nocc)
    if foo is None:
        foo, fvv = fock_oo_vv(f, gt, t2, nocc)
    if woooo is None:
        woooo = oooo_block(gt, t2, nocc)
    t = t2
    tx = t2.transpose(0, 1, 3, 2)          # tx[i,j,a,b] = t_ij^ba
    u = 2.0 * t - tx
    r = ein("aibj->ijab", gt[v, o, v, o]).copy()
    # one-body dressing (Fock-like) terms
    r += ein("be,ijae->ijab", fvv, t) + ein("ae,ijeb->ijab", fvv, t)
    r -= ein("mj,imab->ijab", foo, t) + ein("mi,mjab->ijab", foo, t)
    # hole-hole and particle-particle ladders
    r += ein("minj,mnab->ijab", woooo, t)
    r += ein("aebf,ijef->ijab", gt[v, v, v, v], t)
    # linear rings
    g_ovvo = gt[o, v, v, o]   # g[m,e,b,j]
    g_oovv = gt[o, o, v, v]   # g[m,j,b,e]
    r += ein("mebj,imae->ijab", g_ovvo, u)
    r -= ein("mjbe,imae->ijab", g_oovv, t)
    r -= ein("mibe,jmea->ijab", g_oovv, t)
    r -= ein("mjae,imeb->ijab", g_oovv, t)
    r += ein("meai,jmbe->ijab", g_ovvo, u)
    r -= ein("miae,jmbe->ijab", g_oovv, t)
    # quadratic rings
    g_ovov = gt[o, v, o, v]   # g[m,e,n,f]
    r += ein("imae,menf,jnbf->ijab", u, g_ovov, u)
    r -= ein("imae,mfne,jnbf->ijab", u, g_ovov, t)
    r += ein("imae,mfne,jnfb->ijab", t, g_ovov, t)
    r += ein("jmea,mfne,infb->ijab", t, g_ovov, t)
    return r


def hbar2(h: np.ndarray, g: np.ndarray, t1: np.ndarray, t2: np.ndarray, nocc: int):
    """(E0, F[n,n], W[n,n,n,n]) of H-bar_<=2 for the pool (t1, t2)."""
    n = h.shape[0]
    o, v = slice(0, nocc), slice(nocc, n)
    ht, gt = t1_transform(h, g, t1, nocc)
    _, f = reference_terms(ht, gt, nocc)
    t = t2
    tx = t2.transpose(0, 1, 3, 2)
    u = 2.0 * t - tx
    e0 = energy(ht, gt, t2, nocc)

    F = f.copy()
    foo, fvv = fock_oo_vv(f, gt, t2, nocc)
    F[o, o] = foo
    F[v, v] = fvv
    F[v, o] = singles_residual(f, gt, t2, nocc)

    W = gt.copy()
    g_ovov = gt[o, v, o, v]
    # oooo / vvvv
    woooo = oooo_block(gt, t2, nocc)
    W[o, o, o, o] = woooo
    W[v, v, v, v] = gt[v, v, v, v] + ein("menf,mnab->aebf", g_ovov, t)
    # (ov|vo) and its pair partner (vo|ov)
    w_ovvo = gt[o, v, v, o] + ein("menf,jnbf->mebj", g_ovov, u) - ein("mfne,jnbf->mebj", g_ovov, t)
    W[o, v, v, o] = w_ovvo
    W[v, o, o, v] = w_ovvo.transpose(2, 3, 0, 1)
    # (oo|vv) and (vv|oo)
    w_oovv = gt[o, o, v, v] - ein("ifnb,jnfa->ijab", g_ovov, t)
    W[o, o, v, v] = w_oovv
    W[v, v, o, o] = w_oovv.transpose(2, 3, 0, 1)
    # (oo|vo) and (vo|oo)
    w_oovo = (gt[o, o, v, o]
              + ein("me,ijeb->mibj", f[o, v], t)
              + ein("mebf,ijef->mibj", gt[o, v, v, v], t)
              + ein("mine,jnbe->mibj", gt[o, o, o, v], u)
              - ein("meni,jnbe->mibj", gt[o, v, o, o], t)
              - ein("menj,ineb->mibj", gt[o, v, o, o], t))
    W[o, o, v, o] = w_oovo
    W[v, o, o, o] = w_oovo.transpose(2, 3, 0, 1)
    # (vv|vo) and (vo|vv)
    w_vvvo = (gt[v, v, v, o]
              - ein("me,miab->aebi", f[o, v], t)
              + ein("meni,mnab->aebi", gt[o, v, o, o], t)
              + ein("mfae,mifb->aebi", gt[o, v, v, v], u)
              - ein("mebf,miaf->aebi", gt[o, v, v, v], t)
              - ein("meaf,mifb->aebi", gt[o, v, v, v], t))
    W[v, v, v, o] = w_vvvo
    W[v, o, v, v] = w_vvvo.transpose(2, 3, 0, 1)
    # (vo|vo): the doubles residual
    r2 = doubles_residual(f, gt, t2, nocc, foo=foo, fvv=fvv, woooo=woooo)
    W[v, o, v, o] = r2.transpose(2, 0, 3, 1)
    return e0, F, W
