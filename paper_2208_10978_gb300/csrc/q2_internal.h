// Internal definitions shared by the host scheduler and the tile kernels.
//
// Tiling.  A pass works on tiles of 2^T amplitudes.  Its local space is a
// T-dimensional GF(2) subspace W of index space spanned by w_0..w_{T-1},
// with w_b = e_b for b < C (so a tile is made of contiguous 2^C-amplitude
// chunks) and every other w_b free of the low C bits.  Tiles are the cosets
// of W: tile t, local index l is the amplitude
//     i = deposit(t, umask) ^ (XOR_{b: l_b = 1} w_b),
// where umask holds the n - T qubit positions that are not pivots of W.  A
// rotation or Hamiltonian term with xmask x in W maps every tile onto itself,
// so a pass may hold any run of groups whose xmasks span at most T dimensions
// together with e_0..e_{C-1}: one new dimension per new xmask, however many
// qubits that xmask touches.  parity(i & z) = parity(packed & packz(z)) with
// packed = (t << T) | l and packz(z) = (extract(z, umask) << T) |
// sum_b parity(w_b & z) << b.
//
// Groups.  Consecutive rotations with the same xmask and the same parity of
// popcount(x & z) commute (their strings agree on every qubit where both
// have X or Y, and differ on an even number of X/Y-vs-Y/X positions), so on
// each amplitude pair {i, i ^ x} their product is one 2x2 rotation whose
// angle is a signed sum of the group's angles.  The sign pattern depends on
// i only through the parities parity(i & b_l) for a basis b_1..b_r of the
// group's zmasks: the r-bit "code".  A per-group look-up table (LUT) of
// 2^r entries holds cos/sin of the combined angle for every code, computed
// on the host in double precision.  Hamiltonian terms sharing an xmask are
// grouped the same way: the LUT then holds the combined coefficients
// (R, Q) of the pair {i, i^x} for every code.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace q2 {

constexpr int NT = 256;          // threads per CTA of the tile kernels
constexpr int R_MAX = 8;         // max code bits of a Hamiltonian group
constexpr int R_MAX_ROT = 6;     // max code bits of a rotation group (sign masks fit 64 bits)
constexpr int M_MAX = 16;        // max rotations in one rotation group
constexpr int P_MAX = 32;        // max per-thread diagonal iterations over a tile (2^T <= NT * P_MAX)
constexpr int RP_MAX = 512;      // max rotations in one pass (reverse-sweep partials)
constexpr int G_STAGE = 64;      // max groups per pass (staged in shared memory)
constexpr int LUT_STAGE = 1024;  // max LUT entries per pass (staged in shared memory)
constexpr int LUT_STAGE_HAM_C64 = 2048;  // ... for Hamiltonian passes in complex64 (8-byte entries)
constexpr int T_MIN = 8;
constexpr int T_LIMIT = 13;

// Group kinds.  Rotation groups: DIAG (x = 0, a phase per code), REAL (odd
// Y count: real 2x2 rotation of each pair), XROT (even Y count: c - i s X).
// Hamiltonian groups: DIAG, REAL (every member has an even Y count, so the
// pair coefficient R - iQ is real: Q = 0 at every code) and PAIR (general).
enum : uint8_t { KIND_DIAG = 0, KIND_REAL = 1, KIND_XROT = 2, KIND_PAIR = 3 };

constexpr int D_MAX = 4;         // max span dimension of a register block (rotations)
constexpr int D_MAX_EXPECT = 3;  // max span dimension of a Hamiltonian register block

// Register blocks.  Consecutive groups of a pass whose xmasks span d <= D_MAX
// local dimensions form a block.  The block's span V has as basis v_1..v_d
// the groups' own xmasks in order of appearance (so a group that opens a
// dimension pairs along one basis bit); the pivots are the highest bits of
// V's echelon rows, on which the basis is invertible.  V splits a tile into
// 2^(T-d) cosets; thread tid takes cosets s = tid + NT*j, whose amplitudes
// are the local indices base(s) ^ comb[c] (c < 2^d), base(s) = s with zero
// bits inserted at the pivots.  A thread keeps one coset in registers while
// it applies every group of the block; a group with xmask coordinates a in V
// pairs combo c with c ^ a.  A block is canonical (BlockDesc::canon = d)
// when its first d groups pair along bits 0..d-1 and are REAL; kernels
// unroll those.  The code of an amplitude is the XOR of a tile part
// (computed once per tile) and host-tabulated parts for the lane, the warp,
// the coset j and the combo c, all linear in the local index.  Group LUTs
// start at multiples of their 2^r entries (passes at multiples of the
// largest), so kernels reach an entry by XOR of the code into its offset.
struct alignas(16) GroupDesc {
  uint64_t bp[R_MAX];      // code basis in packed-index space
  uint32_t xl;             // xmask in local-index space (0 for diagonal groups)
  uint32_t lut;            // first LUT entry of this group
  uint32_t rot0;           // rotation groups: first rotation, relative to the pass
  uint8_t kind;            // KIND_*
  uint8_t r;               // code bits; the LUT has 2^r entries
  uint8_t m;               // rotation groups: number of rotations
  uint8_t a;               // xmask coordinates in its block's basis (0: diagonal)
  // block enumeration (sweep, expectation)
  uint8_t bjcode[16];      // code of coset offset uj[j]
  uint8_t bccode[16];      // code of combo offset comb[c]
  uint8_t blane[32];       // code of base(lane)
  uint8_t bwarp[8];        // code of base(32 * warp)
  // pair enumeration (H apply, reverse sweep): pair q = tid + NT*j is local
  // index insert_zero(q, pivot), partner ^ xl; diagonal groups use l = tid + NT*j
  uint8_t pivot;           // highest bit of xl
  uint8_t one_param;       // rotation groups: every rotation shares one parameter (reverse sweep
                           // accumulates dE/dtheta of the group with the weights at wlut)
  uint8_t pad0[2];
  uint32_t wlut;           // first entry of the group's gradient weights (2^r entries)
  uint8_t pjcode[32];      // code of the j-th per-thread offset
  uint8_t plane[32];       // code of the lane part of the thread's first element
  uint8_t pwarp[8];        // code of the warp part
  uint16_t pu[16];         // local offset of pair j for thread 0: insert_zero(NT*j, pivot)
  uint8_t pad1[8];
};
static_assert(sizeof(GroupDesc) == 272, "GroupDesc layout");

struct alignas(16) BlockDesc {
  uint16_t comb[16];       // local offset of combo c (c < 2^d)
  uint16_t uj[16];         // local offset of coset j for thread 0: base(NT * j)
  uint8_t d;               // span dimension, 1..D_MAX
  uint8_t piv[D_MAX];      // pivots, ascending
  uint8_t canon;           // number of leading groups k = 0..canon-1 with a = 1 << k and real
                           // pair coefficients (REAL kind), unrolled with fixed pair offsets
  uint8_t pad0[2];
  uint16_t g_begin, g_end; // groups of the block, relative to the pass
  uint8_t pad1[4];
};
static_assert(sizeof(BlockDesc) == 80, "BlockDesc layout");

struct PassDesc {
  uint64_t w[T_LIMIT];    // local basis; w[b] = e_b for b < C
  uint64_t umask;         // tile-index qubit positions
  int T;                  // local dimension
  int C;                  // chunk = 2^C contiguous amplitudes
  int g_begin, g_end;     // groups [g_begin, g_end)
  int rot_begin, rot_end; // rotation plans: rotations covered by this pass
  int lut_begin, lut_count;  // LUT entries of this pass's groups (contiguous)
  int b_begin, b_end;     // register blocks [b_begin, b_end)
};

// Host-side schedule of a rotation list (an ansatz or one apply call).
struct RotPlan {
  int n = 0;
  int T = 0;
  std::vector<PassDesc> passes;
  std::vector<GroupDesc> groups;       // device image
  std::vector<BlockDesc> blocks;
  std::vector<int> grp_rot_begin;      // rotations of group g: [begin, begin + m)
  std::vector<uint8_t> rot_coord;      // per rotation: z_k in the group's code basis
  std::vector<int8_t> rot_sigma;       // per rotation: fixed sign of its angle in the LUT
  std::vector<uint64_t> signmask;      // per rotation: bit c set iff its sign at code c is -1
  int64_t lut_entries = 0;
  int max_pass_rots = 0;
  // Gradient weights of one-parameter groups: w_g(code) = sum_k coef_k sign_k(code)
  // (set by set_param_weights), and per rotation the factor that folds its
  // reverse-sweep sum into dE/dtheta: coef_k for rotations of other groups, 1 for
  // the first rotation of a one-parameter group (its sum already carries the
  // coefficients) and 0 for the group's other rotations.
  std::vector<double> wlut;
  std::vector<double> fold;
  std::vector<uint8_t> pass_one_param;   // every group of the pass is a one-parameter group
  // Every block of the pass is canonical, 4-dimensional and holds exactly its four
  // pairing groups (the sweep's fast path), and the pass has at most 16 groups.
  std::vector<uint8_t> pass_canon4;
  // LUT of (cos b, sin b) for every group and code, b = sum_k sign_k(code) phi_k / 2.
  void build_lut(const double *phi, double *lut2) const;
};

// Host-side schedule of a Hamiltonian.
struct HamPlan {
  int n = 0;
  int T = 0;
  std::vector<PassDesc> passes;
  std::vector<GroupDesc> groups;
  std::vector<BlockDesc> blocks;
  std::vector<double> lut2;            // (R, Q) per group and code
  int64_t lut_entries = 0;
  // Terms of each group: indices term_idx[term_begin[g] .. term_begin[g + 1]) of the
  // Hamiltonian's term arrays (groups as stored, i.e. after block reordering).
  std::vector<int64_t> term_idx;
  std::vector<int64_t> term_begin;
  // Every group of the pass is REAL or DIAG and every block has at most 3
  // dimensions (the expectation's lean path).
  std::vector<uint8_t> pass_lean;
  // Device image of the LUT for the lean path in single precision: (R, R) for REAL
  // and DIAG groups (whose Q is 0), (R, Q) otherwise.
  std::vector<float> lut_f32() const;
};

// Keep only the passes that shard `shard` of `n_shards` evaluates: passes are
// dealt to shards largest first (work = pair evaluations per amplitude, a
// diagonal group counting twice, plus one for the state read), each to the
// least loaded shard (ties: lower pass index, lower shard index).
void restrict_to_shard(HamPlan &p, int shard, int n_shards);

RotPlan build_rot_plan(int n, int64_t n_rot, const uint64_t *x, const uint64_t *z, int T, int C);
void set_param_weights(RotPlan &p, const int32_t *param, const double *coef);
HamPlan build_ham_plan(int n, int64_t n_terms, const uint64_t *x, const uint64_t *z,
                       const double *c, int T, int C, int lut_stage = LUT_STAGE);
int64_t count_x_groups(int64_t n_terms, const uint64_t *x);

// ---- bit helpers (host and device)
#if defined(__CUDACC__)
#define Q2_HD __host__ __device__ __forceinline__
#else
#define Q2_HD inline
#endif

Q2_HD uint64_t deposit_bits(uint64_t v, uint64_t mask) {
  uint64_t out = 0;
  while (mask) {
    uint64_t low = mask & (~mask + 1);
    if (v & 1) out |= low;
    v >>= 1;
    mask &= mask - 1;
  }
  return out;
}

Q2_HD uint64_t extract_bits(uint64_t v, uint64_t mask) {
  uint64_t out = 0;
  int k = 0;
  while (mask) {
    uint64_t low = mask & (~mask + 1);
    if (v & low) out |= (uint64_t)1 << k;
    ++k;
    mask &= mask - 1;
  }
  return out;
}

Q2_HD uint32_t insert_zero(uint32_t q, int p) {
  uint32_t lo = q & ((1u << p) - 1u);
  return ((q >> p) << (p + 1)) | lo;
}

}  // namespace q2
