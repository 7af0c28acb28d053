"""Block-sparse application of the site matrix Theta_c (oracle; test infrastructure).

The paper cuts its contractions into quantum-number slices (Sec. III): with
charge-conserving tensors every contraction splits into independent products of
charge blocks, and each output block is computed by one task that sums the
block products feeding it, so no two tasks write the same output. This module
restates the application Y = Theta_c X of the zip-up (Sec. IV, contraction
pattern 2(a): boundary x vectors, the site sandwich, environment x vectors)
for the vectors of one sector in that form, with the dense FP64 sandwich
C[L, U, R, Dn] of ``oracle.network`` as the site tensor, and returns the task
list with it, so that a block-sparse GPU path can be checked task by task;
``theta_t_blocks`` does the same for the transpose application Theta_c^T, and
``theta_r_blocks`` / ``theta_r_t_blocks`` for the right-environment map of the
CBE fit and its transpose (the four site maps of the path).

Charges are pairs (N_up, N_dn), with the rules of ``oracle.symmetric``:
  boundary tensor T[t, U, t']:   q_t = Q_U + q_t'
  sandwich C[L, U, R, Dn]:       Q_L + Q_U = Q_R + Q_Dn
  left environment EL[a, t, L]:  q_a = q_t + Q_L
  vectors of sector q:           X[t', R, k] nonzero only where q_t' + Q_R = q,
                                 Y[a, Dn, k] nonzero only where q_a - Q_Dn = q.
The three steps and their tasks (one per output block, keyed by its charges):
  1. G1[t, U, R] = sum_t' T[t, U, t'] X[t', R]: block (q_t, Q_U, Q_R) from the
     single t' block q_t' = q_t - Q_U (then Q_R = q - q_t');
  2. G2[t, L, Dn] = sum_{U, R} C[L, U, R, Dn] G1[t, U, R]: block (q_t, Q_L, Q_Dn),
     q_t + Q_L - Q_Dn = q, summed over the U blocks with R = Q_U + Q_L - Q_Dn;
  3. Y[a, Dn] = sum_{t, L} EL[a, t, L] G2[t, L, Dn]: block (q_a, Q_Dn),
     q_a - Q_Dn = q, summed over the (q_t, Q_L) blocks with q_t + Q_L = q_a.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .network import sandwich_full


def charge_groups(q: np.ndarray) -> dict:
    """Index lists of every charge on a leg: {(N_up, N_dn): ascending indices}."""
    out: dict = {}
    for i, x in enumerate(np.asarray(q).reshape(-1, 2).tolist()):
        out.setdefault(tuple(x), []).append(i)
    return {k: np.array(v) for k, v in out.items()}


def _add(a, b):
    return (a[0] + b[0], a[1] + b[1])


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1])


def _accumulate(acc, p):
    """Sum of the block products of one task."""
    return p if acc is None else acc + p


@dataclasses.dataclass
class Task:
    step: int          # 1: boundary x vectors, 2: sandwich, 3: environment x vectors
    out: tuple         # charges of the output block
    terms: int         # block products summed into it
    flops: float       # 2 x multiply-adds of those products


def theta_blocks(EL, qa, T, qt, qU, qtp, A, W, qsite, X, q):
    """Y = Theta_c X by charge blocks for the vectors X[t', R, k] of sector q.

    EL[a, t, L] with bond charges qa (a) and qt (t); T[t, U, t'] with qt, qU, qtp;
    qsite = (Q_L, Q_U, Q_R, Q_Dn) of the site's bundles (Q_U must equal qU).
    Returns (Y [a, Dn, k], tasks)."""
    q = tuple(q)
    C = sandwich_full(A, W)
    QL, QU, QR, QD = qsite
    gA, gT, gTp = charge_groups(qa), charge_groups(qt), charge_groups(qtp)
    gL, gU, gR, gD = charge_groups(QL), charge_groups(QU), charge_groups(QR), charge_groups(QD)
    k = X.shape[2]
    tasks = []
    # 1. boundary x vectors
    G1 = np.zeros((T.shape[0], T.shape[1], X.shape[1], k))
    for ctp, itp in gTp.items():
        cr = _sub(q, ctp)
        if cr not in gR:
            continue
        ir = gR[cr]
        for cu, iu in gU.items():
            ct = _add(cu, ctp)
            if ct not in gT:
                continue
            it = gT[ct]
            blk = np.einsum("tUs,sRk->tURk", T[np.ix_(it, iu, itp)], X[np.ix_(itp, ir)], optimize=True)
            G1[np.ix_(it, iu, ir)] = blk
            tasks.append(Task(1, (ct, cu, cr), 1, 2.0 * len(it) * len(iu) * len(itp) * len(ir) * k))
    # 2. the site sandwich
    G2 = np.zeros((T.shape[0], C.shape[0], C.shape[3], k))
    for ct, it in gT.items():
        for cl, il in gL.items():
            cd = _sub(_add(ct, cl), q)
            if cd not in gD:
                continue
            idd = gD[cd]
            acc, terms, fl = None, 0, 0.0
            for cu, iu in gU.items():
                cr = _sub(_add(cu, cl), cd)
                if cr not in gR:
                    continue
                ir = gR[cr]
                p = np.einsum("LURD,tURk->tLDk", C[np.ix_(il, iu, ir, idd)], G1[np.ix_(it, iu, ir)], optimize=True)
                acc = _accumulate(acc, p)
                terms += 1
                fl += 2.0 * len(it) * len(il) * len(iu) * len(ir) * len(idd) * k
            if acc is not None:
                G2[np.ix_(it, il, idd)] = acc
                tasks.append(Task(2, (ct, cl, cd), terms, fl))
    # 3. environment x vectors
    Y = np.zeros((EL.shape[0], C.shape[3], k))
    for ca, ia in gA.items():
        cd = _sub(ca, q)
        if cd not in gD:
            continue
        idd = gD[cd]
        acc, terms, fl = None, 0, 0.0
        for ct, it in gT.items():
            cl = _sub(ca, ct)
            if cl not in gL:
                continue
            il = gL[cl]
            p = np.einsum("atL,tLDk->aDk", EL[np.ix_(ia, it, il)], G2[np.ix_(it, il, idd)], optimize=True)
            acc = _accumulate(acc, p)
            terms += 1
            fl += 2.0 * len(ia) * len(it) * len(il) * len(idd) * k
        if acc is not None:
            Y[np.ix_(ia, idd)] = acc
            tasks.append(Task(3, (ca, cd), terms, fl))
    return Y, tasks


def theta_t_blocks(EL, qa, T, qt, qU, qtp, A, W, qsite, Y, q):
    """Z = Theta_c^T Y by charge blocks for the vectors Y[a, Dn, k] of sector q (q_a - Q_Dn = q).
    The mirror of theta_blocks (the transpose application of the rSVD, Sec. IV):
      1. H1[t, L, Dn] = sum_a EL[a, t, L] Y[a, Dn]: block (q_t, Q_L, Q_Dn), q_t + Q_L - Q_Dn = q,
         from the single a block q_a = q_t + Q_L;
      2. H2[t, U, R] = sum_{L, Dn} C[L, U, R, Dn] H1[t, L, Dn]: block (q_t, Q_U, Q_R),
         q_t - Q_U + Q_R = q, summed over the L blocks with Dn = L + U - R;
      3. Z[t', R] = sum_{t, U} T[t, U, t'] H2[t, U, R]: block (q_t', Q_R), q_t' + Q_R = q,
         summed over the U blocks with t = U + t'.
    Returns (Z [t', R, k], tasks)."""
    q = tuple(q)
    C = sandwich_full(A, W)
    QL, QU, QR, QD = qsite
    gA, gT, gTp = charge_groups(qa), charge_groups(qt), charge_groups(qtp)
    gL, gU, gR, gD = charge_groups(QL), charge_groups(QU), charge_groups(QR), charge_groups(QD)
    k = Y.shape[2]
    tasks = []
    # 1. environment^T x vectors
    H1 = np.zeros((T.shape[0], C.shape[0], C.shape[3], k))
    for ct, it in gT.items():
        for cl, il in gL.items():
            ca = _add(ct, cl)
            cd = _sub(ca, q)
            if ca not in gA or cd not in gD:
                continue
            ia, idd = gA[ca], gD[cd]
            H1[np.ix_(it, il, idd)] = np.einsum("atL,aDk->tLDk", EL[np.ix_(ia, it, il)], Y[np.ix_(ia, idd)],
                                                optimize=True)
            tasks.append(Task(1, (ct, cl, cd), 1, 2.0 * len(ia) * len(it) * len(il) * len(idd) * k))
    # 2. the site sandwich, transposed
    H2 = np.zeros((T.shape[0], C.shape[1], C.shape[2], k))
    for ct, it in gT.items():
        for cu, iu in gU.items():
            cr = _add(_sub(q, ct), cu)
            if cr not in gR:
                continue
            ir = gR[cr]
            acc, terms, fl = None, 0, 0.0
            for cl, il in gL.items():
                cd = _sub(_add(cl, cu), cr)
                if cd not in gD:
                    continue
                idd = gD[cd]
                p = np.einsum("LURD,tLDk->tURk", C[np.ix_(il, iu, ir, idd)], H1[np.ix_(it, il, idd)], optimize=True)
                acc = _accumulate(acc, p)
                terms += 1
                fl += 2.0 * len(it) * len(il) * len(iu) * len(ir) * len(idd) * k
            if acc is not None:
                H2[np.ix_(it, iu, ir)] = acc
                tasks.append(Task(2, (ct, cu, cr), terms, fl))
    # 3. boundary^T x vectors
    Z = np.zeros((T.shape[2], C.shape[2], k))
    for ctp, itp in gTp.items():
        cr = _sub(q, ctp)
        if cr not in gR:
            continue
        ir = gR[cr]
        acc, terms, fl = None, 0, 0.0
        for cu, iu in gU.items():
            ct = _add(cu, ctp)
            if ct not in gT:
                continue
            it = gT[ct]
            p = np.einsum("tUs,tURk->sRk", T[np.ix_(it, iu, itp)], H2[np.ix_(it, iu, ir)], optimize=True)
            acc = _accumulate(acc, p)
            terms += 1
            fl += 2.0 * len(it) * len(iu) * len(itp) * len(ir) * k
        if acc is not None:
            Z[np.ix_(itp, ir)] = acc
            tasks.append(Task(3, (ctp, cr), terms, fl))
    return Z, tasks


def theta_r_blocks(ER, qa, T, qt, qU, qtp, A, W, qsite, X, q):
    """Z = ThetaR_c X by charge blocks (the right-environment map of the CBE fit, Sec. IV / Fig. 5)
    for the vectors X[Dn, a, k] of sector q, with the right environment ER[a, t', R]:
      ER: q_a = q_t' + Q_R;  X in sector q: Q_Dn + q_a = q;  Z[t, L] in sector q: q_t + Q_L = q.
      1. W1[t', R, Dn] = sum_a ER[a, t', R] X[Dn, a]: block (q_t', Q_R, Q_Dn), one a block;
      2. W2[t', L, U] = sum_{R, Dn} C[L, U, R, Dn] W1[t', R, Dn]: block (q_t', Q_L, Q_U), summed
         over the R blocks with Dn = L + U - R;
      3. Z[t, L] = sum_{t', U} T[t, U, t'] W2[t', L, U]: block (q_t, Q_L), summed over the U blocks
         with t' = t - U.
    Returns (Z [t, L, k], tasks)."""
    q = tuple(q)
    C = sandwich_full(A, W)
    QL, QU, QR, QD = qsite
    gA, gT, gTp = charge_groups(qa), charge_groups(qt), charge_groups(qtp)
    gL, gU, gR, gD = charge_groups(QL), charge_groups(QU), charge_groups(QR), charge_groups(QD)
    k = X.shape[2]
    tasks = []
    W1 = np.zeros((T.shape[2], C.shape[2], C.shape[3], k))
    for ctp, itp in gTp.items():
        for cr, ir in gR.items():
            ca = _add(ctp, cr)
            cd = _sub(q, ca)
            if ca not in gA or cd not in gD:
                continue
            ia, idd = gA[ca], gD[cd]
            W1[np.ix_(itp, ir, idd)] = np.einsum("asR,Dak->sRDk", ER[np.ix_(ia, itp, ir)], X[np.ix_(idd, ia)],
                                                 optimize=True)
            tasks.append(Task(1, (ctp, cr, cd), 1, 2.0 * len(ia) * len(itp) * len(ir) * len(idd) * k))
    W2 = np.zeros((T.shape[2], C.shape[0], C.shape[1], k))
    for ctp, itp in gTp.items():
        for cl, il in gL.items():
            cu = _sub(_sub(q, ctp), cl)
            if cu not in gU:
                continue
            iu = gU[cu]
            acc, terms, fl = None, 0, 0.0
            for cr, ir in gR.items():
                cd = _sub(_add(cl, cu), cr)
                if cd not in gD:
                    continue
                idd = gD[cd]
                p = np.einsum("LURD,sRDk->sLUk", C[np.ix_(il, iu, ir, idd)], W1[np.ix_(itp, ir, idd)], optimize=True)
                acc = _accumulate(acc, p)
                terms += 1
                fl += 2.0 * len(itp) * len(il) * len(iu) * len(ir) * len(idd) * k
            if acc is not None:
                W2[np.ix_(itp, il, iu)] = acc
                tasks.append(Task(2, (ctp, cl, cu), terms, fl))
    Z = np.zeros((T.shape[0], C.shape[0], k))
    for ct, it in gT.items():
        cl = _sub(q, ct)
        if cl not in gL:
            continue
        il = gL[cl]
        acc, terms, fl = None, 0, 0.0
        for cu, iu in gU.items():
            ctp = _sub(ct, cu)
            if ctp not in gTp:
                continue
            itp = gTp[ctp]
            p = np.einsum("tUs,sLUk->tLk", T[np.ix_(it, iu, itp)], W2[np.ix_(itp, il, iu)], optimize=True)
            acc = _accumulate(acc, p)
            terms += 1
            fl += 2.0 * len(it) * len(iu) * len(itp) * len(il) * k
        if acc is not None:
            Z[np.ix_(it, il)] = acc
            tasks.append(Task(3, (ct, cl), terms, fl))
    return Z, tasks


def theta_r_t_blocks(ER, qa, T, qt, qU, qtp, A, W, qsite, Z, q):
    """X = ThetaR_c^T Z by charge blocks for the vectors Z[t, L, k] of sector q (q_t + Q_L = q):
      1. V1[t', L, U] = sum_t T[t, U, t'] Z[t, L]: block (q_t', Q_L, Q_U), one t block t = U + t';
      2. V2[t', R, Dn] = sum_{L, U} C[L, U, R, Dn] V1[t', L, U]: block (q_t', Q_R, Q_Dn), summed
         over the L blocks with U = R + Dn - L;
      3. X[Dn, a] = sum_{t', R} ER[a, t', R] V2[t', R, Dn]: block (Q_Dn, q_a), summed over the t'
         blocks with R = a - t'.
    Returns (X [Dn, a, k], tasks)."""
    q = tuple(q)
    C = sandwich_full(A, W)
    QL, QU, QR, QD = qsite
    gA, gT, gTp = charge_groups(qa), charge_groups(qt), charge_groups(qtp)
    gL, gU, gR, gD = charge_groups(QL), charge_groups(QU), charge_groups(QR), charge_groups(QD)
    k = Z.shape[2]
    tasks = []
    V1 = np.zeros((T.shape[2], C.shape[0], C.shape[1], k))
    for ctp, itp in gTp.items():
        for cl, il in gL.items():
            cu = _sub(_sub(q, ctp), cl)
            ct = _add(cu, ctp)
            if cu not in gU or ct not in gT:
                continue
            iu, it = gU[cu], gT[ct]
            V1[np.ix_(itp, il, iu)] = np.einsum("tUs,tLk->sLUk", T[np.ix_(it, iu, itp)], Z[np.ix_(it, il)],
                                                optimize=True)
            tasks.append(Task(1, (ctp, cl, cu), 1, 2.0 * len(it) * len(iu) * len(itp) * len(il) * k))
    V2 = np.zeros((T.shape[2], C.shape[2], C.shape[3], k))
    for ctp, itp in gTp.items():
        for cr, ir in gR.items():
            cd = _sub(_sub(q, ctp), cr)
            if cd not in gD:
                continue
            idd = gD[cd]
            acc, terms, fl = None, 0, 0.0
            for cl, il in gL.items():
                cu = _sub(_add(cr, cd), cl)
                if cu not in gU:
                    continue
                iu = gU[cu]
                p = np.einsum("LURD,sLUk->sRDk", C[np.ix_(il, iu, ir, idd)], V1[np.ix_(itp, il, iu)], optimize=True)
                acc = _accumulate(acc, p)
                terms += 1
                fl += 2.0 * len(itp) * len(il) * len(iu) * len(ir) * len(idd) * k
            if acc is not None:
                V2[np.ix_(itp, ir, idd)] = acc
                tasks.append(Task(2, (ctp, cr, cd), terms, fl))
    X = np.zeros((C.shape[3], ER.shape[0], k))
    for cd, idd in gD.items():
        ca = _sub(q, cd)
        if ca not in gA:
            continue
        ia = gA[ca]
        acc, terms, fl = None, 0, 0.0
        for ctp, itp in gTp.items():
            cr = _sub(ca, ctp)
            if cr not in gR:
                continue
            ir = gR[cr]
            p = np.einsum("asR,sRDk->Dak", ER[np.ix_(ia, itp, ir)], V2[np.ix_(itp, ir, idd)], optimize=True)
            acc = _accumulate(acc, p)
            terms += 1
            fl += 2.0 * len(ia) * len(itp) * len(ir) * len(idd) * k
        if acc is not None:
            X[np.ix_(idd, ia)] = acc
            tasks.append(Task(3, (cd, ca), terms, fl))
    return X, tasks


def dense_flops(EL, T, A, W, X) -> float:
    """Multiply-add count x 2 of the same three steps with dense tensors (no blocks)."""
    C = sandwich_full(A, W)
    t, u, tp = T.shape
    r, k = X.shape[1], X.shape[2]
    a, l, d = EL.shape[0], C.shape[0], C.shape[3]
    return 2.0 * k * (t * u * tp * r + t * l * u * r * d + a * t * l * d)
