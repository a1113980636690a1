// Term generator for the excitation classes A-G (host code).
//
// A product of spin-free generators E_pq = sum_s a+_ps a_qs between reference
// states with a doubly occupied core and an empty virtual space splits into
// closed, virtual and active fermion strings (the reordering sign is the parity
// of the stable partition).  Closed strings are fully contracted against the
// filled core (only creator-left pairs survive), virtual strings against the empty
// space (only annihilator-left pairs), and the active string is brought to normal
// order with a_p a+_q = delta_pq - a+_q a_p.  Each contraction identifies the spin
// variables of its two operators; a spin variable left on no operator sums to 2,
// and in the normal-ordered active string every creator pairs with the annihilator
// carrying its spin variable, which gives the spin-free RDM
// Gamma_{p1q1,...,pkqk} = <M| sum a+_p1 .. a+_pk a_qk .. a_q1 |N> and a permutation sign.
#include "terms.h"

#include <algorithm>
#include <map>
#include <numeric>
#include <stdexcept>
#include <tuple>
#include <utility>

namespace caspt2 {
namespace {

// ------------------------------------------------------------------ classes (Eq. class)
// slot ids inside a class; families list the slots of p, q, r, s in E_{pq,rs}
const ClassDef kClasses[7] = {
    // A: E_ri,st          slots r i s t
    {1, {{0, 1, 2, 3}, {0, 0, 0, 0}}, 4, {SP_A, SP_C, SP_A, SP_A}, 1, {1, 0, 0}, 3, {0, 2, 3}, -1, -1},
    // B: E_ri,sj          slots r i s j
    {1, {{0, 1, 2, 3}, {0, 0, 0, 0}}, 4, {SP_A, SP_C, SP_A, SP_C}, 2, {1, 3, 0}, 2, {0, 2, 0}, 1, 3},
    // C: E_ar,st          slots a r s t
    {1, {{0, 1, 2, 3}, {0, 0, 0, 0}}, 4, {SP_V, SP_A, SP_A, SP_A}, 1, {0, 0, 0}, 3, {1, 2, 3}, -1, -1},
    // D: E_ai,rs + E_ar,si  slots a i r s
    {2, {{0, 1, 2, 3}, {0, 2, 3, 1}}, 4, {SP_V, SP_C, SP_A, SP_A}, 2, {0, 1, 0}, 2, {2, 3, 0}, -1, -1},
    // E: E_ai,rj          slots a i r j
    {1, {{0, 1, 2, 3}, {0, 0, 0, 0}}, 4, {SP_V, SP_C, SP_A, SP_C}, 3, {0, 1, 3}, 1, {2, 0, 0}, 1, 3},
    // F: E_ar,bs          slots a r b s
    {1, {{0, 1, 2, 3}, {0, 0, 0, 0}}, 4, {SP_V, SP_A, SP_V, SP_A}, 2, {0, 2, 0}, 2, {1, 3, 0}, 0, 2},
    // G: E_ar,bi          slots a r b i
    {1, {{0, 1, 2, 3}, {0, 0, 0, 0}}, 4, {SP_V, SP_A, SP_V, SP_C}, 3, {0, 2, 3}, 1, {1, 0, 0}, 0, 2},
};

// ------------------------------------------------------------------ fermion algebra
struct FOp {
  bool cre;
  int lab;
  int spin;
};

struct Contracted {
  int sign;
  std::vector<std::pair<int, int>> deltas;  // label pairs
  std::vector<std::pair<int, int>> merges;  // spin variable pairs
};

// complete pairings of a closed (filled, creator-left) or virtual (empty,
// annihilator-left) string
void pairings(const std::vector<FOp>& ops, bool creator_left, std::vector<Contracted>& out) {
  if (ops.empty()) {
    out.push_back({1, {}, {}});
    return;
  }
  if (ops.size() % 2 || ops[0].cre != creator_left) return;
  for (size_t k = 1; k < ops.size(); ++k) {
    if (ops[k].cre == ops[0].cre) continue;
    std::vector<FOp> rest(ops.begin() + 1, ops.begin() + k);
    rest.insert(rest.end(), ops.begin() + k + 1, ops.end());
    std::vector<Contracted> sub;
    pairings(rest, creator_left, sub);
    const int sg = ((k - 1) % 2) ? -1 : 1;
    for (auto& c : sub) {
      c.sign *= sg;
      c.deltas.insert(c.deltas.begin(), {ops[0].lab, ops[k].lab});
      c.merges.insert(c.merges.begin(), {ops[0].spin, ops[k].spin});
      out.push_back(std::move(c));
    }
  }
}

struct Ordered {
  int coeff;
  std::vector<std::pair<int, int>> deltas, merges;
  std::vector<FOp> ops;
};

void normal_order(const std::vector<FOp>& ops, std::vector<Ordered>& out) {
  for (size_t i = 0; i + 1 < ops.size(); ++i) {
    if (!ops[i].cre && ops[i + 1].cre) {
      std::vector<FOp> sw = ops;
      std::swap(sw[i], sw[i + 1]);
      std::vector<Ordered> a;
      normal_order(sw, a);
      for (auto& t : a) {
        t.coeff = -t.coeff;
        out.push_back(std::move(t));
      }
      std::vector<FOp> ct(ops.begin(), ops.begin() + i);
      ct.insert(ct.end(), ops.begin() + i + 2, ops.end());
      std::vector<Ordered> b;
      normal_order(ct, b);
      for (auto& t : b) {
        t.deltas.insert(t.deltas.begin(), {ops[i].lab, ops[i + 1].lab});
        t.merges.insert(t.merges.begin(), {ops[i].spin, ops[i + 1].spin});
        out.push_back(std::move(t));
      }
      return;
    }
  }
  out.push_back({1, {}, {}, ops});
}

int perm_sign(std::vector<int> p) {
  int s = 1;
  for (size_t i = 0; i < p.size(); ++i)
    while (p[i] != (int)i) {
      std::swap(p[i], p[p[i]]);
      s = -s;
    }
  return s;
}

struct UnionFind {
  std::map<int, int> par;
  int find(int x) {
    if (!par.count(x)) par[x] = x;
    while (par[x] != x) x = par[x] = par[par[x]];
    return x;
  }
  void join(int a, int b) {
    int ra = find(a), rb = find(b);
    if (ra != rb) par[ra] = rb;
  }
};

using Key = std::pair<std::vector<std::pair<int, int>>, std::vector<std::pair<int, int>>>;

// <M| ops |N> reduced to {(deltas, rdm pairs) -> coefficient}
std::map<Key, long> reduce(const std::vector<FOp>& ops, const std::map<int, Space>& space) {
  std::vector<int> order(ops.size());
  std::iota(order.begin(), order.end(), 0);
  auto rank = [&](int i) {
    Space s = space.at(ops[i].lab);
    return s == SP_C ? 0 : (s == SP_V ? 1 : 2);
  };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return rank(x) < rank(y); });
  const int sign0 = perm_sign(order);
  std::vector<FOp> core, virt, act;
  std::vector<int> spins;
  for (int i : order) {
    const FOp& o = ops[i];
    spins.push_back(o.spin);
    Space s = space.at(o.lab);
    (s == SP_C ? core : (s == SP_V ? virt : act)).push_back(o);
  }
  std::vector<Contracted> pc, pv;
  pairings(core, true, pc);
  pairings(virt, false, pv);
  std::vector<Ordered> na;
  normal_order(act, na);
  std::map<Key, long> acc;
  for (const auto& c1 : pc)
    for (const auto& c2 : pv)
      for (const auto& c3 : na) {
        UnionFind uf;
        for (auto* m : {&c1.merges, &c2.merges, &c3.merges})
          for (auto& pr : *m) uf.join(pr.first, pr.second);
        std::vector<FOp> cre, ann;
        for (const auto& o : c3.ops) (o.cre ? cre : ann).push_back(o);
        if (cre.size() != ann.size()) continue;
        std::map<int, int> live;
        for (const auto& o : c3.ops) live[uf.find(o.spin)] = 1;
        std::map<int, int> all;
        for (int s : spins) all[uf.find(s)] = 1;
        const long nfree = (long)all.size() - (long)live.size();
        const int k = (int)cre.size();
        std::vector<int> target(k, -1);
        for (int j = 0; j < k; ++j) {
          int hits = 0;
          for (int t = 0; t < k; ++t)
            if (uf.find(ann[t].spin) == uf.find(cre[j].spin)) {
              target[j] = t;
              ++hits;
            }
          if (hits != 1) throw std::logic_error("unpaired spin class");
        }
        std::vector<int> perm(k);
        for (int j = 0; j < k; ++j) perm[k - 1 - j] = target[j];
        Key key;
        for (auto* d : {&c1.deltas, &c2.deltas, &c3.deltas})
          for (auto pr : *d) key.first.push_back(std::minmax(pr.first, pr.second));
        std::sort(key.first.begin(), key.first.end());
        for (int j = 0; j < k; ++j) key.second.push_back({cre[j].lab, ann[target[j]].lab});
        acc[key] += (long)sign0 * c1.sign * c2.sign * c3.coeff * perm_sign(perm) * (1L << nfree);
      }
  return acc;
}

struct OpBuilder {
  int next_spin = 0;
  void E(std::vector<FOp>& v, int p, int q) {
    int s = next_spin++;
    v.push_back({true, p, s});
    v.push_back({false, q, s});
  }
  void E2(std::vector<FOp>& v, int p, int q, int r, int t) {  // E_{pq,rt}
    int s = next_spin++, u = next_spin++;
    v.push_back({true, p, s});
    v.push_back({true, r, u});
    v.push_back({false, t, u});
    v.push_back({false, q, s});
  }
};

// labels: bra slots 0..3, ket slots 4..7, f indices 8, 9, Hamiltonian indices 10..13
constexpr int kLabKet = 4, kLabU = 8, kLabW = 9, kLabH = 10;

}  // namespace

const ClassDef& class_def(int cls) { return kClasses[cls]; }

void build_act_plans(int cls, bool with_fock, std::vector<ActPlan>& out) {
  const ClassDef& C = kClasses[cls];
  std::map<int, Space> sp;
  for (int s = 0; s < C.nslot; ++s) sp[s] = sp[kLabKet + s] = C.slot_space[s];
  sp[kLabU] = sp[kLabW] = SP_A;
  auto is_ext = [&](int lab) { return lab < 8 && C.slot_space[lab % 4] != SP_A; };
  for (int fb = 0; fb < C.nfam; ++fb)
    for (int fk = 0; fk < C.nfam; ++fk) {
      std::vector<FOp> ops;
      OpBuilder b;
      const int* pb = C.fam[fb];
      const int* pk = C.fam[fk];
      b.E2(ops, pb[1], pb[0], pb[3], pb[2]);  // (E_{pq,rs})^dagger = E_{qp,sr}
      if (with_fock) b.E(ops, kLabU, kLabW);
      b.E2(ops, kLabKet + pk[0], kLabKet + pk[1], kLabKet + pk[2], kLabKet + pk[3]);
      for (const auto& kv : reduce(ops, sp)) {
        if (kv.second == 0) continue;
        ActPlan P{};
        P.coeff = (double)kv.second;
        P.fb = fb;
        P.fk = fk;
        P.has_f = with_fock ? 1 : 0;
        // external pattern
        int map_to[4] = {-1, -1, -1, -1};
        UnionFind uf;
        for (auto d : kv.first.first) {
          if (is_ext(d.first)) {
            int x = d.first, y = d.second;
            if (x >= kLabKet) std::swap(x, y);
            map_to[x] = y - kLabKet;
          } else {
            uf.join(d.first, d.second);
          }
        }
        bool ident = true, swapped = C.pair0 >= 0;
        for (int e = 0; e < C.next; ++e) {
          int s = C.ext[e];
          if (map_to[s] != s) ident = false;
          int want = s == C.pair0 ? C.pair1 : (s == C.pair1 ? C.pair0 : s);
          if (map_to[s] != want) swapped = false;
        }
        if (!ident && !swapped) throw std::logic_error("unexpected external pattern");
        P.pi = ident ? 0 : 1;
        // active label classes -> references
        std::map<int, int> ref;   // root -> ref
        auto out_ref = [&](int lab) -> int {
          for (int k = 0; k < C.nact; ++k) {
            if (lab == C.act[k]) return kRefBra + k;
            if (lab == kLabKet + C.act[k]) return kRefKet + k;
          }
          return -1;
        };
        std::vector<int> labs;
        for (int k = 0; k < C.nact; ++k) labs.push_back(C.act[k]);
        for (int k = 0; k < C.nact; ++k) labs.push_back(kLabKet + C.act[k]);
        if (with_fock) {
          labs.push_back(kLabU);
          labs.push_back(kLabW);
        }
        for (int lab : labs) {
          int r = uf.find(lab), o = out_ref(lab);
          if (o < 0) continue;
          if (!ref.count(r)) {
            ref[r] = o;
          } else {
            P.eq[P.neq][0] = ref[r];
            P.eq[P.neq][1] = o;
            ++P.neq;
          }
        }
        for (int lab : labs) {
          int r = uf.find(lab);
          if (!ref.count(r)) ref[r] = kRefLoop + P.nloop++;
        }
        const auto& rd = kv.first.second;
        P.rank = (int8_t)rd.size();
        for (size_t j = 0; j < rd.size(); ++j) {
          P.idx[2 * j] = ref.at(uf.find(rd[j].first));
          P.idx[2 * j + 1] = ref.at(uf.find(rd[j].second));
        }
        if (with_fock) {
          P.fidx[0] = ref.at(uf.find(kLabU));
          P.fidx[1] = ref.at(uf.find(kLabW));
        }
        out.push_back(P);
      }
    }
}

void build_src_plans(int cls, std::vector<SrcPlan>& out) {
  const ClassDef& C = kClasses[cls];
  const Space spaces[3] = {SP_C, SP_A, SP_V};
  for (int fb = 0; fb < C.nfam; ++fb) {
    for (int kind = 0; kind < 2; ++kind) {
      const int nh = kind == 0 ? 2 : 4;
      int ncomb = kind == 0 ? 9 : 81;
      for (int comb = 0; comb < ncomb; ++comb) {
        Space hs[4];
        int cc = comb;
        for (int k = nh - 1; k >= 0; --k) {
          hs[k] = spaces[cc % 3];
          cc /= 3;
        }
        std::map<int, Space> sp;
        for (int s = 0; s < C.nslot; ++s) sp[s] = C.slot_space[s];
        for (int k = 0; k < nh; ++k) sp[kLabH + k] = hs[k];
        std::vector<FOp> ops;
        OpBuilder b;
        const int* pb = C.fam[fb];
        b.E2(ops, pb[1], pb[0], pb[3], pb[2]);
        if (kind == 0)
          b.E(ops, kLabH, kLabH + 1);
        else
          b.E2(ops, kLabH, kLabH + 1, kLabH + 2, kLabH + 3);
        for (const auto& kv : reduce(ops, sp)) {
          if (kv.second == 0) continue;
          SrcPlan P{};
          P.coeff = (double)kv.second * (kind == 1 ? 0.5 : 1.0);
          P.fb = fb;
          P.kind = kind;
          UnionFind uf;
          for (auto d : kv.first.first) uf.join(d.first, d.second);
          std::map<int, int> ref;
          for (int s = 0; s < C.nslot; ++s) {  // outputs: every bra slot
            int r = uf.find(s);
            if (!ref.count(r)) {
              ref[r] = kRefBra + s;
            } else {
              P.eq[P.neq][0] = ref[r];
              P.eq[P.neq][1] = kRefBra + s;
              ++P.neq;
            }
          }
          for (int k = 0; k < nh; ++k) {
            int r = uf.find(kLabH + k);
            if (!ref.count(r)) {
              P.loop_space[P.nloop] = hs[k];
              ref[r] = kRefLoop + P.nloop++;
            }
          }
          int ii[4];
          Space is[4];
          for (int k = 0; k < nh; ++k) {
            ii[k] = ref.at(uf.find(kLabH + k));
            is[k] = hs[k];
          }
          // canonical integral block: h_pq = h_qp, (pq|rt) = (qp|rt) = (rt|pq)
          if (is[0] > is[1]) { std::swap(is[0], is[1]); std::swap(ii[0], ii[1]); }
          if (kind == 1) {
            if (is[2] > is[3]) { std::swap(is[2], is[3]); std::swap(ii[2], ii[3]); }
            if (std::make_pair(is[0], is[1]) > std::make_pair(is[2], is[3])) {
              std::swap(is[0], is[2]); std::swap(ii[0], ii[2]);
              std::swap(is[1], is[3]); std::swap(ii[1], ii[3]);
            }
          }
          for (int k = 0; k < nh; ++k) {
            P.iidx[k] = ii[k];
            P.ispace[k] = is[k];
          }
          const auto& rd = kv.first.second;
          P.rank = (int8_t)rd.size();
          for (size_t j = 0; j < rd.size(); ++j) {
            P.idx[2 * j] = ref.at(uf.find(rd[j].first));
            P.idx[2 * j + 1] = ref.at(uf.find(rd[j].second));
          }
          out.push_back(P);
        }
      }
    }
  }
}

void split_src_plans(int cls, const std::vector<SrcPlan>& in, std::vector<SrcPlan>& rest,
                     std::vector<SrcGemmGroup>& groups) {
  const ClassDef& C = kClasses[cls];
  rest.clear();
  groups.clear();
  auto is_bra = [](int r) { return r >= kRefBra && r < kRefBra + 8; };
  auto slot_sp = [&](int r) { return C.slot_space[r - kRefBra]; };
  for (const SrcPlan& P : in) {
    const int ni = P.kind == 0 ? 2 : 4;
    bool ok = true;
    for (int j = 0; j < ni; ++j)
      if (is_bra(P.iidx[j]) && slot_sp(P.iidx[j]) == SP_A) ok = false;
    int cls_of[4] = {0, 0, 0, 0};          // 1 shared, 2 integral-only, 3 RDM-only
    for (int j = 0; j < P.nloop && ok; ++j) {
      bool inI = false, inR = false;
      for (int q = 0; q < ni; ++q) inI = inI || P.iidx[q] == kRefLoop + j;
      for (int q = 0; q < 2 * P.rank; ++q) inR = inR || P.idx[q] == kRefLoop + j;
      for (int q = 0; q < P.neq; ++q)
        if (P.eq[q][0] == kRefLoop + j || P.eq[q][1] == kRefLoop + j) ok = false;
      cls_of[j] = inI && inR ? 1 : (inI ? 2 : (inR ? 3 : 0));
      if (cls_of[j] == 0) ok = false;
      if ((cls_of[j] == 1 || cls_of[j] == 3) && P.loop_space[j] != SP_A) ok = false;
    }
    if (!ok) {
      rest.push_back(P);
      continue;
    }
    // canonical numbering: shared and RDM-only loops by first appearance in the RDM
    // indices, integral-only loops in order
    int pos[4] = {-1, -1, -1, -1};
    int ns = 0, nr = 0, nx = 0;
    for (int q = 0; q < 2 * P.rank; ++q) {
      const int r = P.idx[q];
      if (r >= kRefLoop && r < kRefLoop + 4 && cls_of[r - kRefLoop] == 1 && pos[r - kRefLoop] < 0)
        pos[r - kRefLoop] = ns++;
    }
    for (int q = 0; q < 2 * P.rank; ++q) {
      const int r = P.idx[q];
      if (r >= kRefLoop && r < kRefLoop + 4 && cls_of[r - kRefLoop] == 3 && pos[r - kRefLoop] < 0)
        pos[r - kRefLoop] = nr++;
    }
    for (int j = 0; j < P.nloop; ++j)
      if (cls_of[j] == 2) pos[j] = nx++;
    if (ns > 2 || nr > 3) {
      rest.push_back(P);
      continue;
    }
    auto gref = [&](int r) -> int8_t {
      if (r >= kRefLoop && r < kRefLoop + 4) {
        const int j = r - kRefLoop;
        return (int8_t)(kRefLoop + (cls_of[j] == 1 ? pos[j] : ns + pos[j]));
      }
      return (int8_t)r;
    };
    SrcGSig g{};
    g.rank = P.rank;
    g.ns = (int8_t)ns;
    g.nloop = (int8_t)nr;
    for (int q = 0; q < 2 * P.rank; ++q) g.idx[q] = gref(P.idx[q]);
    SrcXTerm x{};
    x.coeff = P.coeff;
    x.kind = P.kind;
    x.cb = P.cb;
    for (int q = 0; q < 4; ++q) {
      x.ispace[q] = P.ispace[q];
      x.iidx[q] = q < ni ? gref(P.iidx[q]) : 0;
    }
    x.nloop = (int8_t)nx;
    for (int j = 0; j < P.nloop; ++j)
      if (cls_of[j] == 2) x.loop_space[pos[j]] = P.loop_space[j];
    for (int q = 0; q < P.neq; ++q) {
      const int r0 = P.eq[q][0], r1 = P.eq[q][1];
      if (slot_sp(r0) == SP_A) {
        g.eq[g.neq][0] = (int8_t)std::min(r0, r1);
        g.eq[g.neq][1] = (int8_t)std::max(r0, r1);
        ++g.neq;
      } else {
        x.eq[x.neq][0] = (int8_t)r0;
        x.eq[x.neq][1] = (int8_t)r1;
        ++x.neq;
      }
    }
    bool placed = false;
    for (SrcGemmGroup& G : groups) {
      if (G.fb != P.fb || G.g.rank != g.rank || G.g.ns != g.ns || G.g.nloop != g.nloop ||
          G.g.neq != g.neq)
        continue;
      bool same = true;
      for (int q = 0; q < 2 * g.rank && same; ++q) same = G.g.idx[q] == g.idx[q];
      for (int q = 0; q < g.neq && same; ++q)
        same = G.g.eq[q][0] == g.eq[q][0] && G.g.eq[q][1] == g.eq[q][1];
      if (same) {
        G.x.push_back(x);
        placed = true;
        break;
      }
    }
    if (!placed) groups.push_back(SrcGemmGroup{P.fb, g, {x}});
  }
}

void presum_src_plans(const std::vector<SrcPlan>& in, std::vector<SrcPlan>& out,
                      std::vector<PresumSpec>& specs) {
  out.clear();
  for (const SrcPlan& P : in) {
    if (P.kind != 1 || P.nloop == 0) {
      out.push_back(P);
      continue;
    }
    // loop variables that appear only in the integral can be summed inside it
    bool summable[4] = {true, true, true, true};
    for (int j = 0; j < 2 * P.rank; ++j)
      if (P.idx[j] >= kRefLoop) summable[P.idx[j] - kRefLoop] = false;
    for (int q = 0; q < P.neq; ++q)
      for (int r = 0; r < 2; ++r)
        if (P.eq[q][r] >= kRefLoop) summable[P.eq[q][r] - kRefLoop] = false;
    int svar[4] = {-1, -1, -1, -1}, nsv = 0;
    for (int j = 0; j < P.nloop; ++j)
      if (summable[j]) svar[j] = nsv++;
    if (nsv == 0 || nsv > 2) {
      out.push_back(P);
      continue;
    }
    PresumSpec sp{};
    SrcPlan Q = P;
    Q.kind = 2;
    int newloop[4] = {-1, -1, -1, -1}, nl = 0;
    for (int j = 0; j < P.nloop; ++j)
      if (!summable[j]) {
        newloop[j] = nl;
        Q.loop_space[nl++] = P.loop_space[j];
      }
    for (int j = nl; j < 4; ++j) Q.loop_space[j] = 0;
    Q.nloop = (int8_t)nl;
    auto remap = [&](int8_t ref) -> int8_t {
      if (ref < kRefLoop) return ref;
      return (int8_t)(kRefLoop + newloop[ref - kRefLoop]);
    };
    for (int p = 0; p < 4; ++p) {
      sp.space[p] = P.ispace[p];
      const int ref = P.iidx[p];
      if (ref >= kRefLoop && summable[ref - kRefLoop]) {
        sp.var[p] = (int8_t)svar[ref - kRefLoop];
        Q.iidx[p] = kRefZero;
        Q.ispace[p] = kSpUnit;
      } else {
        sp.var[p] = -1;
        Q.iidx[p] = remap(P.iidx[p]);
      }
    }
    for (int j = 0; j < 2 * P.rank; ++j) Q.idx[j] = remap(P.idx[j]);
    int id = -1;
    for (size_t k = 0; k < specs.size(); ++k)
      if (specs[k] == sp) id = (int)k;
    if (id < 0) {
      id = (int)specs.size();
      specs.push_back(sp);
    }
    Q.cb = (int8_t)id;
    out.push_back(Q);
  }
}

namespace {
// class H for the couplings: E_ai,bj, slots a i b j; external positions i, j, a, b
const ClassDef kClassH = {1, {{0, 1, 2, 3}, {0, 0, 0, 0}}, 4, {SP_V, SP_C, SP_V, SP_C}, 3,
                          {1, 3, 0}, 0, {0, 0, 0}, -1, -1};
const int kHExt[4] = {1, 3, 0, 2};
const ClassDef& xdef(int cls) { return cls == 7 ? kClassH : kClasses[cls]; }
int xnext(int cls) { return cls == 7 ? 4 : kClasses[cls].next; }
int xext(int cls, int k) { return cls == 7 ? kHExt[k] : kClasses[cls].ext[k]; }
// (closed holes, virtual particles) of each class
const int kCount[8][2] = {{1, 0}, {2, 0}, {0, 1}, {1, 1}, {2, 1}, {0, 2}, {1, 2}, {2, 2}};
constexpr int kLabX = 8, kLabY = 9;
}  // namespace

XClassInfo xclass_info(int cls) {
  const ClassDef& C = xdef(cls);
  XClassInfo I{};
  I.nfam = C.nfam;
  I.next = xnext(cls);
  I.nact = C.nact;
  for (int k = 0; k < I.next; ++k) I.ext_space[k] = C.slot_space[xext(cls, k)];
  return I;
}

void build_cross_groups(int X, int Y, std::vector<CrossGroup>& out) {
  const int dh = (Y == SP_C) - (X == SP_C), dp = (X == SP_V) - (Y == SP_V);
  for (int Kp = 0; Kp < 8; ++Kp) {
    int K = -1;
    for (int q = 0; q < 8; ++q)
      if (kCount[q][0] == kCount[Kp][0] + dh && kCount[q][1] == kCount[Kp][1] + dp) K = q;
    if (K < 0) continue;
    const ClassDef& CB = xdef(K);
    const ClassDef& CK = xdef(Kp);
    std::map<int, Space> sp;
    for (int s = 0; s < 4; ++s) {
      sp[s] = CB.slot_space[s];
      sp[kLabKet + s] = CK.slot_space[s];
    }
    sp[kLabX] = (Space)X;
    sp[kLabY] = (Space)Y;
    auto bra_pos = [&](int lab) {          // external position of a bra slot label
      for (int k = 0; k < xnext(K); ++k)
        if (xext(K, k) == lab) return k;
      return -1;
    };
    auto ket_pos = [&](int lab) {
      for (int k = 0; k < xnext(Kp); ++k)
        if (kLabKet + xext(Kp, k) == lab) return k;
      return -1;
    };
    auto act_ref = [&](int lab) -> int {
      for (int k = 0; k < CB.nact; ++k)
        if (lab == CB.act[k]) return kRefBra + k;
      for (int k = 0; k < CK.nact; ++k)
        if (lab == kLabKet + CK.act[k]) return kRefKet + k;
      if ((lab == kLabX && X == SP_A) || (lab == kLabY && Y == SP_A)) return kRefT;
      return -1;
    };
    const size_t first = out.size();
    for (int fb = 0; fb < CB.nfam; ++fb)
      for (int fk = 0; fk < CK.nfam; ++fk) {
        std::vector<FOp> ops;
        OpBuilder b;
        const int* pb = CB.fam[fb];
        const int* pk = CK.fam[fk];
        b.E2(ops, pb[1], pb[0], pb[3], pb[2]);      // (E_{pq,rs})^dagger = E_{qp,sr}
        b.E(ops, kLabX, kLabY);
        b.E2(ops, kLabKet + pk[0], kLabKet + pk[1], kLabKet + pk[2], kLabKet + pk[3]);
        for (const auto& kv : reduce(ops, sp)) {
          if (kv.second == 0) continue;
          CrossGroup g{};
          g.K = K;
          g.Kp = Kp;
          g.X = X;
          g.Y = Y;
          g.t_xy = X == SP_A ? 0 : (Y == SP_A ? 1 : -1);
          for (int k = 0; k < 4; ++k) g.ket_src[k] = -1;
          g.side = -1;
          UnionFind uf;
          for (auto d : kv.first.first) {
            const int l0 = d.first, l1 = d.second;
            if (sp.at(l0) == SP_A) {
              uf.join(l0, l1);
              continue;
            }
            // external delta: bra-ket, bra-f or ket-f
            int lb = -1, lk = -1, lf = -1;
            for (int l : {l0, l1}) {
              if (l == kLabX || l == kLabY) lf = l;
              else if (l >= kLabKet) lk = l;
              else lb = l;
            }
            if (lb >= 0 && lk >= 0) {
              g.ket_src[ket_pos(lk)] = bra_pos(lb);
            } else if (lf >= 0 && (lb >= 0 || lk >= 0)) {
              const int side = lb >= 0 ? 0 : 1;
              if (g.side >= 0 && g.side != side) throw std::logic_error("mixed external sides");
              g.side = side;
              g.fe_xy[g.nfe] = lf == kLabX ? 0 : 1;
              g.fe_pos[g.nfe] = side == 0 ? bra_pos(lb) : ket_pos(lk);
              ++g.nfe;
            } else {
              throw std::logic_error("unexpected external delta");
            }
          }
          if (g.nfe == 0 || g.side < 0) throw std::logic_error("f index not external");
          if (g.nfe == 2 && g.fe_xy[0] == 1) {        // x first
            std::swap(g.fe_xy[0], g.fe_xy[1]);
            std::swap(g.fe_pos[0], g.fe_pos[1]);
          }
          CrossPlan P{};
          P.coeff = (double)kv.second;
          P.fb = (int8_t)fb;
          P.fk = (int8_t)fk;
          std::vector<int> labs;
          for (int k = 0; k < CB.nact; ++k) labs.push_back(CB.act[k]);
          for (int k = 0; k < CK.nact; ++k) labs.push_back(kLabKet + CK.act[k]);
          if (g.t_xy >= 0) labs.push_back(g.t_xy == 0 ? kLabX : kLabY);
          std::map<int, int> ref;
          for (int lab : labs) {
            const int r = uf.find(lab), o = act_ref(lab);
            if (!ref.count(r)) {
              ref[r] = o;
            } else {
              if (P.neq >= 6) throw std::logic_error("too many active equalities");
              P.eq[P.neq][0] = (int8_t)ref[r];
              P.eq[P.neq][1] = (int8_t)o;
              ++P.neq;
            }
          }
          const auto& rd = kv.first.second;
          if (rd.size() > 4) throw std::logic_error("RDM rank above 4");
          P.rank = (int8_t)rd.size();
          for (size_t j = 0; j < rd.size(); ++j) {
            P.idx[2 * j] = (int8_t)ref.at(uf.find(rd[j].first));
            P.idx[2 * j + 1] = (int8_t)ref.at(uf.find(rd[j].second));
          }
          // append to the group with the same pattern
          bool placed = false;
          for (size_t q = first; q < out.size() && !placed; ++q) {
            CrossGroup& h = out[q];
            bool same = h.side == g.side && h.nfe == g.nfe;
            for (int k = 0; k < g.nfe && same; ++k)
              same = h.fe_xy[k] == g.fe_xy[k] && h.fe_pos[k] == g.fe_pos[k];
            for (int k = 0; k < 4 && same; ++k) same = h.ket_src[k] == g.ket_src[k];
            if (same) {
              h.terms.push_back(P);
              placed = true;
            }
          }
          if (!placed) {
            g.terms.push_back(P);
            out.push_back(std::move(g));
          }
        }
      }
  }
}

}  // namespace caspt2
