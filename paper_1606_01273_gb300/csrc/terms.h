// Contraction terms of the excitation classes (host-side generator; not part of the C ABI).
//
// The overlap, active-Fock and source matrix elements of every class in Eq. (class)
// are products of spin-free generators between reference states whose closed
// orbitals are doubly occupied and whose virtual orbitals are empty.  The generator
// reduces each product to active-space RDMs and emits "access plans": for every term,
// which RDM rank and which output / loop index feeds each RDM index, which integral
// block and indices multiply it, and which index equalities it requires.  The device
// kernels in class_ag.cu evaluate these plans.
#pragma once
#include <cstdint>
#include <vector>

namespace caspt2 {

enum Space : int8_t { SP_C = 0, SP_A = 1, SP_V = 2 };

// An index reference in a plan: output bra slot k (k < 8), output ket slot (8 + k),
// or loop variable (16 + k).
constexpr int kRefBra = 0, kRefKet = 8, kRefLoop = 16;

struct ClassDef {
  int nfam;            // operator families (class D has two)
  int fam[2][4];       // slot ids of p, q, r, s in E_{pq,rs}
  int nslot;
  Space slot_space[4];
  int next, ext[3];    // external slots in output order
  int nact, act[3];    // active slots in output order
  int pair0, pair1;    // external slots that can be swapped (-1 if none)
};

const ClassDef& class_def(int cls);   // cls = 0..6 for classes A..G

// Term of S / F_act: coeff * [prod eq] * sum_{loops} f[l0][l1]^{has_f} * Gamma_rank[idx...]
// indices refer to bra active slots, ket active slots or loop variables (all active).
struct ActPlan {
  double coeff;
  int8_t fb, fk, pi, rank, has_f, nloop, neq;
  int8_t idx[8];       // RDM indices p1 q1 p2 q2 ... (refs)
  int8_t fidx[2];      // f indices (refs) when has_f
  int8_t eq[4][2];     // pairs of output refs that must be equal
};

// Term of the sources V[fam][ext...][act...][M][L] = <M|E_Omega^dag H|L>:
// coeff * integral[iidx...] * Gamma_rank[idx...] summed over loop variables.
struct SrcPlan {
  double coeff;        // includes the 1/2 of the two-body part
  int8_t fb, kind;     // kind 0: h_pq, 1: (pq|rt), 2: (pq|rt) pre-summed over loop indices
  int8_t cb;           // kind 2: index of the pre-summed block (see PresumSpec)
  int8_t ispace[4];    // spaces of the integral indices
  int8_t iidx[4];      // integral indices (refs: bra slot = ext/act slot id, loops)
  int8_t rank, nloop, neq;
  int8_t idx[8];
  int8_t loop_space[4];
  int8_t eq[4][2];
};

// A (pq|rt) block summed over loop indices that appear only in the integral (not in an
// RDM index): out[i0][i1][i2][i3] with the summed positions of size 1 (space kSpUnit),
//   out = sum over the loop values of (pq|rt) with the summed positions set to them.
// var[p] = -1 (position kept) or the summed variable (0 or 1; one variable may fill two
// positions, as in sum_j (ij|jr)).
constexpr int kSpUnit = 3;          // extra "space" of dimension 1
constexpr int kRefZero = 23;        // index reference whose value is always 0
struct PresumSpec {
  int8_t space[4];                  // spaces of the source block's positions
  int8_t var[4];
  bool operator==(const PresumSpec& o) const {
    for (int k = 0; k < 4; ++k)
      if (space[k] != o.space[k] || var[k] != o.var[k]) return false;
    return true;
  }
};
// Rewrite the two-electron source plans whose loop indices appear only in the integral
// as kind-2 plans on pre-summed blocks (specs appended to / shared through `specs`).
void presum_src_plans(const std::vector<SrcPlan>& in, std::vector<SrcPlan>& out,
                      std::vector<PresumSpec>& specs);

// Source terms recast as matrix products.  A term whose integral carries only external
// slots and loop indices (no active output slot) factorises as
//   V[fam][ext][(act..., M, L)] += sum_k X[ext][k] G[k][(act..., M, L)],
// k running over the loop indices shared by the integral and the RDM: X = coeff x integral
// (summed over integral-only loops, Kronecker deltas among external slots), G = RDM (summed
// over RDM-only loops, deltas among active slots).  Terms with the same G are grouped and
// their X summed, so a group is one GEMM with K = a^ns.
struct SrcXTerm {
  double coeff;
  int8_t kind, cb;
  int8_t ispace[4];
  int8_t iidx[4];      // refs: bra slots, kRefLoop + p (shared, p < ns), kRefLoop + ns + q
                       // (integral-only loop q), kRefZero
  int8_t nloop;        // integral-only loops
  int8_t loop_space[4];
  int8_t neq;          // deltas among external slots
  int8_t eq[4][2];
};
struct SrcGSig {
  int8_t rank, ns, nloop, neq;  // nloop: RDM-only loops (active)
  int8_t idx[8];                // refs: bra active slots, kRefLoop + p (shared), kRefLoop + ns + q
  int8_t eq[4][2];              // deltas among active slots
};
struct SrcGemmGroup {
  int fb;
  SrcGSig g;
  std::vector<SrcXTerm> x;
};
// Split the (pre-summed) source plans of class cls into GEMM groups and the terms that stay
// with the plan interpreter.
void split_src_plans(int cls, const std::vector<SrcPlan>& in, std::vector<SrcPlan>& rest,
                     std::vector<SrcGemmGroup>& groups);

// Build the plans of class cls (0..6).  Deterministic; a few hundred terms.
void build_act_plans(int cls, bool with_fock, std::vector<ActPlan>& out);
void build_src_plans(int cls, std::vector<SrcPlan>& out);

// ------------------------------------------------------------------ one-body couplings
// <M~| E_bra(K)^dag E_xy E_ket(K') |N~> for x, y in different orbital spaces (closed-active,
// active-virtual, closed-virtual and the transposes): the operator E_xy changes the (closed
// holes, virtual particles) count of a function of class K' into that of class K.  Classes
// 0..6 are A..G (ClassDef), 7 is H (E_ai,bj, external slots in the order i, j, a, b).
// Every closed or virtual index of a term is tied by one Kronecker delta to exactly one
// other, so a term factorises into an external pattern (which bra slot, ket slot or f
// index each external index is tied to) and an active factor (deltas among the bra and ket
// active slots and the active one of x, y, times one RDM).  Terms are grouped by pattern.
constexpr int kRefT = 24;           // index reference of the active one of x, y
struct CrossPlan {                  // the active factor of one term
  double coeff;
  int8_t fb, fk, rank, neq;
  int8_t idx[8];                    // RDM indices (refs: kRefBra + k, kRefKet + k, kRefT)
  int8_t eq[6][2];
};
struct CrossGroup {
  int K, Kp;                        // bra and ket class (0..7)
  int X, Y;                         // spaces of x and y
  int side;                         // 0: the external f indices are tied to bra slots, 1: ket
  int nfe;                          // external f indices (1 or 2)
  int fe_xy[2];                     // 0: x, 1: y
  int fe_pos[2];                    // their bra (side 0) or ket (side 1) external positions
  int t_xy;                         // which of x, y is active (-1: none)
  int ket_src[4];                   // per ket external position: the bra position tied to it,
                                    // or -1 (tied to an f index)
  std::vector<CrossPlan> terms;
};
struct XClassInfo {                 // layout facts of a class for the couplings
  int nfam, next, nact;
  int ext_space[4];                 // spaces of the external positions (output order)
};
XClassInfo xclass_info(int cls);    // cls 0..7
// All groups of the couplings through E_xy with x in space X, y in space Y (X != Y).
void build_cross_groups(int X, int Y, std::vector<CrossGroup>& out);

}  // namespace caspt2
