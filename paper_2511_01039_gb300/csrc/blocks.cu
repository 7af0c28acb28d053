// Task tables of the block-sparse site maps (Theta_c, its transpose, the right-environment map of
// the CBE fit and its transpose; host code).
//
// With charge-conserving tensors every contraction of the application (Sec. IV,
// pattern 2(a) of Sec. III: boundary x vectors, the site sandwich, environment x
// vectors) splits into products of charge blocks; the paper cuts them into
// quantum-number slices whose outputs do not overlap. One task per output block
// sums the block products that feed it, so the tasks of one step can run
// concurrently (one grouped launch) without write conflicts. The table depends
// on the leg charges only; the block kernels that execute it are the next step
// of the charge-sector mode.
//
// Charge rules (pairs (N_up, N_dn)):
//   T[t, U, t']      q_t = Q_U + q_t'
//   C[L, U, R, Dn]   Q_L + Q_U = Q_R + Q_Dn
//   EL[a, t, L]      q_a = q_t + Q_L
//   vectors of sector q: X[t', R] with q_t' + Q_R = q, Y[a, Dn] with q_a - Q_Dn = q.
#include <cstdint>
#include <map>
#include <utility>
#include <vector>

#include "common.cuh"

namespace fpeps {
namespace {

using Q = std::pair<int32_t, int32_t>;

// charges of a leg in the order of their first appearance, with the size of each group
struct Groups {
  std::vector<Q> order;
  std::map<Q, int64_t> size;
  bool has(const Q& q) const { return size.count(q) != 0; }
  int64_t n(const Q& q) const {
    auto it = size.find(q);
    return it == size.end() ? 0 : it->second;
  }
};

Groups groups_of(const int32_t* q, int32_t n) {
  Groups g;
  for (int32_t i = 0; i < n; ++i) {
    const Q c{q[2 * i], q[2 * i + 1]};
    if (!g.size.count(c)) g.order.push_back(c);
    ++g.size[c];
  }
  return g;
}

Q add(const Q& a, const Q& b) { return {a.first + b.first, a.second + b.second}; }
Q sub(const Q& a, const Q& b) { return {a.first - b.first, a.second - b.second}; }

struct BlockTask {
  int32_t step, terms;
  Q out[3];
  double flops;   // 2 x multiply-adds per vector
};

std::vector<BlockTask> theta_tasks(const Groups& gA, const Groups& gT, const Groups& gU, const Groups& gTp,
                                   const Groups& gL, const Groups& gR, const Groups& gD, const Q& q) {
  std::vector<BlockTask> out;
  // 1. G1[t, U, R] = T[t, U, t'] X[t', R]: one t' block per output block
  for (const Q& ctp : gTp.order) {
    const Q cr = sub(q, ctp);
    if (!gR.has(cr)) continue;
    for (const Q& cu : gU.order) {
      const Q ct = add(cu, ctp);
      if (!gT.has(ct)) continue;
      out.push_back({1, 1, {ct, cu, cr}, 2.0 * gT.n(ct) * gU.n(cu) * gTp.n(ctp) * gR.n(cr)});
    }
  }
  // 2. G2[t, L, Dn] = C[L, U, R, Dn] G1[t, U, R], summed over the U blocks with R = U + L - Dn
  for (const Q& ct : gT.order) {
    for (const Q& cl : gL.order) {
      const Q cd = sub(add(ct, cl), q);
      if (!gD.has(cd)) continue;
      BlockTask t{2, 0, {ct, cl, cd}, 0.0};
      for (const Q& cu : gU.order) {
        const Q cr = sub(add(cu, cl), cd);
        if (!gR.has(cr)) continue;
        ++t.terms;
        t.flops += 2.0 * gT.n(ct) * gL.n(cl) * gU.n(cu) * gR.n(cr) * gD.n(cd);
      }
      if (t.terms) out.push_back(t);
    }
  }
  // 3. Y[a, Dn] = EL[a, t, L] G2[t, L, Dn], summed over the (t, L) blocks with t + L = a
  for (const Q& ca : gA.order) {
    const Q cd = sub(ca, q);
    if (!gD.has(cd)) continue;
    BlockTask t{3, 0, {ca, cd, {0, 0}}, 0.0};
    for (const Q& ct : gT.order) {
      const Q cl = sub(ca, ct);
      if (!gL.has(cl)) continue;
      ++t.terms;
      t.flops += 2.0 * gA.n(ca) * gT.n(ct) * gL.n(cl) * gD.n(cd);
    }
    if (t.terms) out.push_back(t);
  }
  return out;
}

// the transpose application Z = Theta_c^T Y (the mirror image: environment^T, sandwich^T, boundary^T)
std::vector<BlockTask> theta_t_tasks(const Groups& gA, const Groups& gT, const Groups& gU, const Groups& gTp,
                                     const Groups& gL, const Groups& gR, const Groups& gD, const Q& q) {
  std::vector<BlockTask> out;
  // 1. H1[t, L, Dn] = EL[a, t, L] Y[a, Dn]: one a block (a = t + L) per output block
  for (const Q& ct : gT.order) {
    for (const Q& cl : gL.order) {
      const Q ca = add(ct, cl), cd = sub(ca, q);
      if (!gA.has(ca) || !gD.has(cd)) continue;
      out.push_back({1, 1, {ct, cl, cd}, 2.0 * gA.n(ca) * gT.n(ct) * gL.n(cl) * gD.n(cd)});
    }
  }
  // 2. H2[t, U, R] = C[L, U, R, Dn] H1[t, L, Dn], summed over the L blocks with Dn = L + U - R
  for (const Q& ct : gT.order) {
    for (const Q& cu : gU.order) {
      const Q cr = add(sub(q, ct), cu);
      if (!gR.has(cr)) continue;
      BlockTask t{2, 0, {ct, cu, cr}, 0.0};
      for (const Q& cl : gL.order) {
        const Q cd = sub(add(cl, cu), cr);
        if (!gD.has(cd)) continue;
        ++t.terms;
        t.flops += 2.0 * gT.n(ct) * gL.n(cl) * gU.n(cu) * gR.n(cr) * gD.n(cd);
      }
      if (t.terms) out.push_back(t);
    }
  }
  // 3. Z[t', R] = T[t, U, t'] H2[t, U, R], summed over the U blocks with t = U + t'
  for (const Q& ctp : gTp.order) {
    const Q cr = sub(q, ctp);
    if (!gR.has(cr)) continue;
    BlockTask t{3, 0, {ctp, cr, {0, 0}}, 0.0};
    for (const Q& cu : gU.order) {
      const Q ct = add(cu, ctp);
      if (!gT.has(ct)) continue;
      ++t.terms;
      t.flops += 2.0 * gT.n(ct) * gU.n(cu) * gTp.n(ctp) * gR.n(cr);
    }
    if (t.terms) out.push_back(t);
  }
  return out;
}

// the right-environment map of the CBE fit, Z[t, L] = ThetaR_c X[Dn, a] with ER[a, t', R]
// (q_a = q_t' + Q_R; X in sector q: Q_Dn + q_a = q)
std::vector<BlockTask> theta_r_tasks(const Groups& gA, const Groups& gT, const Groups& gU, const Groups& gTp,
                                     const Groups& gL, const Groups& gR, const Groups& gD, const Q& q) {
  std::vector<BlockTask> out;
  // 1. W1[t', R, Dn] = ER[a, t', R] X[Dn, a]: one a block (a = t' + R) per output block
  for (const Q& ctp : gTp.order) {
    for (const Q& cr : gR.order) {
      const Q ca = add(ctp, cr), cd = sub(q, ca);
      if (!gA.has(ca) || !gD.has(cd)) continue;
      out.push_back({1, 1, {ctp, cr, cd}, 2.0 * gA.n(ca) * gTp.n(ctp) * gR.n(cr) * gD.n(cd)});
    }
  }
  // 2. W2[t', L, U] = C[L, U, R, Dn] W1[t', R, Dn], summed over the R blocks with Dn = L + U - R
  for (const Q& ctp : gTp.order) {
    for (const Q& cl : gL.order) {
      const Q cu = sub(sub(q, ctp), cl);
      if (!gU.has(cu)) continue;
      BlockTask t{2, 0, {ctp, cl, cu}, 0.0};
      for (const Q& cr : gR.order) {
        const Q cd = sub(add(cl, cu), cr);
        if (!gD.has(cd)) continue;
        ++t.terms;
        t.flops += 2.0 * gTp.n(ctp) * gL.n(cl) * gU.n(cu) * gR.n(cr) * gD.n(cd);
      }
      if (t.terms) out.push_back(t);
    }
  }
  // 3. Z[t, L] = T[t, U, t'] W2[t', L, U], summed over the U blocks with t' = t - U
  for (const Q& ct : gT.order) {
    const Q cl = sub(q, ct);
    if (!gL.has(cl)) continue;
    BlockTask t{3, 0, {ct, cl, {0, 0}}, 0.0};
    for (const Q& cu : gU.order) {
      const Q ctp = sub(ct, cu);
      if (!gTp.has(ctp)) continue;
      ++t.terms;
      t.flops += 2.0 * gT.n(ct) * gU.n(cu) * gTp.n(ctp) * gL.n(cl);
    }
    if (t.terms) out.push_back(t);
  }
  return out;
}

// its transpose, X[Dn, a] = ThetaR_c^T Z[t, L] (Z in sector q: q_t + Q_L = q)
std::vector<BlockTask> theta_r_t_tasks(const Groups& gA, const Groups& gT, const Groups& gU, const Groups& gTp,
                                       const Groups& gL, const Groups& gR, const Groups& gD, const Q& q) {
  std::vector<BlockTask> out;
  // 1. V1[t', L, U] = T[t, U, t'] Z[t, L]: one t block (t = U + t') per output block
  for (const Q& ctp : gTp.order) {
    for (const Q& cl : gL.order) {
      const Q cu = sub(sub(q, ctp), cl), ct = add(cu, ctp);
      if (!gU.has(cu) || !gT.has(ct)) continue;
      out.push_back({1, 1, {ctp, cl, cu}, 2.0 * gT.n(ct) * gU.n(cu) * gTp.n(ctp) * gL.n(cl)});
    }
  }
  // 2. V2[t', R, Dn] = C[L, U, R, Dn] V1[t', L, U], summed over the L blocks with U = R + Dn - L
  for (const Q& ctp : gTp.order) {
    for (const Q& cr : gR.order) {
      const Q cd = sub(sub(q, ctp), cr);
      if (!gD.has(cd)) continue;
      BlockTask t{2, 0, {ctp, cr, cd}, 0.0};
      for (const Q& cl : gL.order) {
        const Q cu = sub(add(cr, cd), cl);
        if (!gU.has(cu)) continue;
        ++t.terms;
        t.flops += 2.0 * gTp.n(ctp) * gL.n(cl) * gU.n(cu) * gR.n(cr) * gD.n(cd);
      }
      if (t.terms) out.push_back(t);
    }
  }
  // 3. X[Dn, a] = ER[a, t', R] V2[t', R, Dn], summed over the t' blocks with R = a - t'
  for (const Q& cd : gD.order) {
    const Q ca = sub(q, cd);
    if (!gA.has(ca)) continue;
    BlockTask t{3, 0, {cd, ca, {0, 0}}, 0.0};
    for (const Q& ctp : gTp.order) {
      const Q cr = sub(ca, ctp);
      if (!gR.has(cr)) continue;
      ++t.terms;
      t.flops += 2.0 * gA.n(ca) * gTp.n(ctp) * gR.n(cr) * gD.n(cd);
    }
    if (t.terms) out.push_back(t);
  }
  return out;
}

}  // namespace
}  // namespace fpeps

extern "C" fpeps_status fpeps_theta_block_tasks(int32_t op, const int32_t* qa, int32_t na, const int32_t* qt, int32_t nt,
                                                const int32_t* qu, int32_t nu, const int32_t* qtp, int32_t ntp,
                                                const int32_t* ql, int32_t nl, const int32_t* qr, int32_t nr,
                                                const int32_t* qd, int32_t nd, const int32_t* q, int32_t* tasks,
                                                double* flops, int32_t* n_inout) {
  if (!qa || !qt || !qu || !qtp || !ql || !qr || !qd || !q || !n_inout) return FPEPS_ERR_ARG;
  if (op < 0 || op > 3) return FPEPS_ERR_ARG;
  if (na < 1 || nt < 1 || nu < 1 || ntp < 1 || nl < 1 || nr < 1 || nd < 1 || *n_inout < 0) return FPEPS_ERR_ARG;
  using namespace fpeps;
  const Groups gA = groups_of(qa, na), gT = groups_of(qt, nt), gU = groups_of(qu, nu), gTp = groups_of(qtp, ntp),
               gL = groups_of(ql, nl), gR = groups_of(qr, nr), gD = groups_of(qd, nd);
  const Q qs{q[0], q[1]};
  const std::vector<BlockTask> tab = op == 0   ? theta_tasks(gA, gT, gU, gTp, gL, gR, gD, qs)
                                     : op == 1 ? theta_t_tasks(gA, gT, gU, gTp, gL, gR, gD, qs)
                                     : op == 2 ? theta_r_tasks(gA, gT, gU, gTp, gL, gR, gD, qs)
                                               : theta_r_t_tasks(gA, gT, gU, gTp, gL, gR, gD, qs);
  const int32_t cap = *n_inout;
  *n_inout = (int32_t)tab.size();
  if (!tasks || !flops) return cap == 0 ? FPEPS_OK : FPEPS_ERR_ARG;
  if (cap < (int32_t)tab.size()) return FPEPS_ERR_ARG;
  for (size_t i = 0; i < tab.size(); ++i) {
    int32_t* o = tasks + 8 * i;
    o[0] = tab[i].step;
    o[1] = tab[i].terms;
    for (int j = 0; j < 3; ++j) {
      o[2 + 2 * j] = tab[i].out[j].first;
      o[3 + 2 * j] = tab[i].out[j].second;
    }
    flops[i] = tab[i].flops;
  }
  return FPEPS_OK;
}
