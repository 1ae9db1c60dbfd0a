// Tile kernels of the state-vector engine (sm_103a).
//
// Every kernel here is HBM-streaming: a persistent grid walks the 2^(n-T)
// tiles of one pass; each CTA brings a tile (2^(T-C) chunks of 2^C
// contiguous amplitudes) into shared memory -- by bulk async copies counted
// on an mbarrier for tiles of 2^9 amplitudes and more, by 16-byte loads
// below that, and by per-thread 16-byte async copies in the two fast kernels
// (k_sweep_c4, k_expect_fast) -- applies all groups of the pass there, and
// writes the tile back (or only reduces it).  Tiles are cosets of the pass's local subspace
// W (see q2_internal.h), so a pass touches every amplitude exactly once and
// tiles never overlap.  The pass's offsets, group and block descriptors and
// LUT are staged in shared memory once per CTA.
//
// The main kernels work on register blocks: for each block of groups whose
// xmasks span d local dimensions, a thread loads a 2^d-amplitude coset into
// registers, applies (or evaluates) every group of the block there with
// compile-time pair indices, and writes it back once.  The fallbacks
// (k_happly, k_reverse) walk one group at a time (pair q = tid + NT*j).
// Codes come from host tables plus one per-tile code per group.
//
//   k_init_hf       HF determinant (Eq. jw-wfn-map)
//   k_sweep         rotation groups in order (product formula after Eq. ucc)
//   k_expect        sum_t c_t <psi|P_t|psi> and <psi|psi> (Eq. qubit-ham-detail)
//   k_happly_blk    lambda = H psi (Algorithm 1, start of the backward pass);
//                   k_happly for tiles below 2^9 amplitudes
//   k_dot           Re<psi|lambda>, <psi|psi>
//   k_reverse_blk   Algorithm 1's reverse loop over one pass of one-parameter
//                   groups (complex64): per-group weighted Im<lambda|P|psi>
//                   sums, then psi and lambda un-rotated together;
//                   k_reverse (per-rotation sums) for every other pass
//   k_reduce_*      fixed-order reductions of per-CTA partials (deterministic)
//   k_wait_probe    the bounded-wait give-up path, for the failure test
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <set>
#include <utility>

#include "q2_internal.h"
#include "kernels.h"

namespace q2 {

template <typename R> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// 16-byte vector of amplitudes: two complex64 or one complex128.
template <typename R> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int amps = 2; };
template <> struct Vec16<double> { using type = double2; static constexpr int amps = 1; };

__device__ __forceinline__ int par64(uint64_t v) { return __popcll(v) & 1; }

template <typename V, bool STREAM>
__device__ __forceinline__ V ld16(const V *p) {
  if constexpr (STREAM) return __ldcs(p);
  else return *p;
}
template <typename V, bool STREAM>
__device__ __forceinline__ void st16(V *p, V v) {
  if constexpr (STREAM) __stcs(p, v);
  else *p = v;
}

// ------------------------------------------------------------------ shared-memory layout

// [tiles: vectors * 2^T amplitudes][off: 2^(T-C) u64][groups][blocks][lut][tcode][extra]
struct SmemLayout {
  size_t tiles, off, groups, blocks, lut, tcode, extra, total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// lut_align: alignment of the staged LUT (bytes, a power of two).  Kernels
// that address a group's LUT by XOR (byte offset | code << log2(entry)) need
// it to be entry bytes << (max code bits); groups start at multiples of 2^r
// entries, so the offset of every group's table then has r free low bits.
__host__ __device__ inline size_t align_to(size_t v, size_t a) { return (v + a - 1) & ~(a - 1); }

__host__ __device__ inline SmemLayout smem_layout(int amp_bytes, const PassDesc &pd, int vectors,
                                                  size_t extra_bytes, int lut_entry_bytes = 0,
                                                  size_t lut_align = 16, size_t lut_slack = 0) {
  if (lut_entry_bytes == 0) lut_entry_bytes = amp_bytes;
  SmemLayout L;
  size_t o = 0;
  L.tiles = o;
  o = align16(o + (size_t)amp_bytes * ((size_t)1 << pd.T) * vectors);
  L.off = o;
  o = align16(o + sizeof(uint64_t) * ((size_t)1 << (pd.T - pd.C)));
  L.groups = o;
  o = align16(o + sizeof(GroupDesc) * (size_t)(pd.g_end - pd.g_begin));
  L.blocks = o;
  o = align16(o + sizeof(BlockDesc) * (size_t)(pd.b_end - pd.b_begin));
  o = align_to(o, lut_align);
  L.lut = o;
  o = align16(o + (size_t)lut_entry_bytes * (size_t)pd.lut_count + lut_slack);
  L.tcode = o;
  o = align16(o + sizeof(uint32_t) * (size_t)(pd.g_end - pd.g_begin));
  L.extra = o;
  o = align16(o + extra_bytes);
  L.total = o;
  return L;
}

// LUT entry of the forward sweep in shared memory.  complex64 with packed
// FP32 pair arithmetic keeps (cos, cos, sin, sin) so both packed operands
// come from one 16-byte load; otherwise (cos, sin).
#ifndef Q2_F32X2
#define Q2_F32X2 1
#endif
template <typename R> struct SweepLut { using E = typename Vec2<R>::type; };
#if Q2_F32X2
template <> struct SweepLut<float> { using E = float4; };
#endif
__device__ __forceinline__ float lut_cos(float2 e) { return e.x; }
__device__ __forceinline__ float lut_sin(float2 e) { return e.y; }
__device__ __forceinline__ double lut_cos(double2 e) { return e.x; }
__device__ __forceinline__ double lut_sin(double2 e) { return e.y; }
__device__ __forceinline__ float lut_cos(float4 e) { return e.x; }
__device__ __forceinline__ float lut_sin(float4 e) { return e.z; }

template <typename R, typename E = typename Vec2<R>::type> struct Stage {
  using C2 = typename Vec2<R>::type;
  int T, C;
  uint32_t amps;
  uint64_t *off;
  const GroupDesc *gs;   // staged groups of the pass (index g - g_begin)
  const BlockDesc *bs;   // staged blocks of the pass (index b - b_begin)
  const E *lut;          // staged LUT, indexed by the global LUT offset
  uint32_t *tcode;       // per-tile code of each group
  const unsigned char *base;   // start of the dynamic shared memory (tile at offset 0)
};

template <typename T>
__device__ __forceinline__ void copy16(void *dst, const T *src, int count) {
  uint4 *d = reinterpret_cast<uint4 *>(dst);
  const uint4 *s = reinterpret_cast<const uint4 *>(src);
  const int n16 = count * (int)(sizeof(T) / 16);
  for (int i = threadIdx.x; i < n16; i += NT) d[i] = __ldg(s + i);
}

// Stage offsets, descriptors and LUT of a pass; caller syncs.
template <typename R, typename E = typename Vec2<R>::type>
__device__ __forceinline__ Stage<R, E> stage_pass(unsigned char *smem, const PassDesc &pd,
                                                  const SmemLayout &L, const GroupDesc *groups,
                                                  const BlockDesc *blocks,
                                                  const typename Vec2<R>::type *lut, uint32_t lut_shift = 0) {
  using C2 = typename Vec2<R>::type;
  Stage<R, E> t;
  t.T = pd.T;
  t.C = pd.C;
  t.amps = 1u << pd.T;
  t.off = reinterpret_cast<uint64_t *>(smem + L.off);
  const int nh = 1 << (pd.T - pd.C);
  for (int h = threadIdx.x; h < nh; h += NT) {
    uint64_t o = 0;
    for (int b = 0; b < pd.T - pd.C; ++b)
      if ((h >> b) & 1) o ^= pd.w[pd.C + b];
    t.off[h] = o;
  }
  copy16(smem + L.groups, groups + pd.g_begin, pd.g_end - pd.g_begin);
  if (blocks) copy16(smem + L.blocks, blocks + pd.b_begin, pd.b_end - pd.b_begin);
  E *ld = reinterpret_cast<E *>(smem + L.lut + lut_shift);
  for (int i = threadIdx.x; i < pd.lut_count; i += NT) {
    const C2 e = __ldg(lut + pd.lut_begin + i);
    if constexpr (sizeof(E) == sizeof(C2)) ld[i] = e;
    else ld[i] = E{e.x, e.x, e.y, e.y};
  }
  t.gs = reinterpret_cast<const GroupDesc *>(smem + L.groups);
  t.bs = reinterpret_cast<const BlockDesc *>(smem + L.blocks);
  t.lut = ld - pd.lut_begin;
  t.base = smem;
  t.tcode = reinterpret_cast<uint32_t *>(smem + L.tcode);
  return t;
}

// Tile part of every group's code for tile t (threads g < ng); caller syncs.
template <typename R, typename E>
__device__ __forceinline__ void tile_codes(const Stage<R, E> &s, int ng, uint64_t t) {
  const int g = threadIdx.x;
  if (g < ng) {
    const GroupDesc &d = s.gs[g];
    const uint64_t packed = t << s.T;
    uint32_t c = 0;
    for (int k = 0; k < d.r; ++k) c |= (uint32_t)par64(packed & d.bp[k]) << k;
    s.tcode[g] = c;
  }
}

__device__ __forceinline__ uint64_t tile_base(uint64_t t, uint64_t umask) { return deposit_bits(t, umask); }

// Tile bases of a persistent CTA (tiles blockIdx.x, + gridDim.x, ...): the
// deposit of t + gridDim.x is the deposit of t plus that of gridDim.x with
// the carry passed across the bits outside the mask, so each step is one add.
struct TileWalk {
  uint64_t base, step, mask;
  __device__ __forceinline__ TileWalk(uint64_t t0, uint64_t stride, uint64_t m)
      : base(deposit_bits(t0, m)), step(deposit_bits(stride, m)), mask(m) {}
  __device__ __forceinline__ void next() { base = ((base | ~mask) + step) & mask; }
};

// Gather one tile of `src` into shared memory (LOAD_BATCH 16-byte loads in flight per thread).
#ifndef Q2_LOAD_BATCH
#define Q2_LOAD_BATCH 4
#endif
constexpr int LOAD_BATCH = Q2_LOAD_BATCH;
template <typename R, bool STREAM, typename E>
__device__ __forceinline__ void load_tile(const R *src, uint64_t base, const Stage<R, E> &tc,
                                          typename Vec16<R>::type *dst) {
  using V = typename Vec16<R>::type;
  constexpr int A = Vec16<R>::amps;
  const uint32_t nv = tc.amps / A;
  const uint32_t cm = (1u << tc.C) - 1u;
  const V *g = reinterpret_cast<const V *>(src);
  for (uint32_t v0 = 0; v0 < nv; v0 += LOAD_BATCH * NT) {
    V buf[LOAD_BATCH];
#pragma unroll
    for (int k = 0; k < LOAD_BATCH; ++k) {
      const uint32_t v = v0 + k * NT + threadIdx.x;
      if (v < nv) {
        const uint32_t l = v * A;
        const uint64_t i = (base ^ tc.off[l >> tc.C]) | (l & cm);
        buf[k] = ld16<V, STREAM>(g + i / A);
      }
    }
#pragma unroll
    for (int k = 0; k < LOAD_BATCH; ++k) {
      const uint32_t v = v0 + k * NT + threadIdx.x;
      if (v < nv) dst[v] = buf[k];
    }
  }
}

template <typename R, bool STREAM, typename E>
__device__ __forceinline__ void store_tile(R *dstg, uint64_t base, const Stage<R, E> &tc,
                                           const typename Vec16<R>::type *src) {
  using V = typename Vec16<R>::type;
  constexpr int A = Vec16<R>::amps;
  const uint32_t nv = tc.amps / A;
  const uint32_t cm = (1u << tc.C) - 1u;
  V *g = reinterpret_cast<V *>(dstg);
#pragma unroll 4
  for (uint32_t v = threadIdx.x; v < nv; v += NT) {
    const uint32_t l = v * A;
    const uint64_t i = (base ^ tc.off[l >> tc.C]) | (l & cm);
    st16<V, STREAM>(g + i / A, src[v]);
  }
}

// ------------------------------------------------------------------ bulk tile copies
//
// Tiles move between HBM and shared memory as 2^C-amplitude chunks (128 bytes
// or more, 16-byte aligned at both ends) by the bulk-copy engine: a thread
// issues one cp.async.bulk per chunk and the CTA waits on an mbarrier that
// counts the bytes, so a CTA waiting for its tile issues no instructions and
// the SM's other CTAs compute meanwhile.  Every wait is bounded: a wait that
// gives up adds one to the calling API function's own fault word (a device
// word that call zeroes before its first launch and reads back with its
// results), and the CTA stops working on its tiles.  Kernels of calls that
// return before their work completes (q2_apply_pauli_rotations,
// q2_apply_hamiltonian) get no fault word and count into g_async_faults,
// which only q2_async_status reads and clears.  The two fast kernels use
// per-thread copies instead (async_load_tile): their waits are hardware
// dependency waits on the thread's own copies, like those of ordinary loads.

__device__ unsigned int g_async_faults;

constexpr uint32_t WAIT_POLLS = 1u << 22;   // try_wait polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bytes to add to region offset `off` of the dynamic shared memory so that the
// region starts at a multiple of `align` (a power of two) in the shared window:
// then a table address that is that start | (index << log2(entry)) is an
// absolute shared address walked by XOR alone.  The layout reserves `align`
// bytes of slack after the region.
__device__ __forceinline__ uint32_t abs_align_shift(const unsigned char *smem, size_t off, size_t align) {
  const uint32_t a = smem_u32(smem + off);
  return (uint32_t)((align - (a & (align - 1))) & (align - 1));
}
__device__ __forceinline__ unsigned long long lds_b64(uint32_t addr) {
  unsigned long long v;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ ulonglong2 lds_b128(uint32_t addr) {
  ulonglong2 v;
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts_b64(uint32_t addr, unsigned long long v) {
  asm volatile("st.shared.b64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *fault,
                                          uint32_t polls = WAIT_POLLS) {
  for (uint32_t i = 0; i < polls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  atomicAdd(fault ? fault : &g_async_faults, 1u);
  return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Start the bulk load of tile `base` (completion counted on bar).
template <typename R, typename E>
__device__ __forceinline__ void bulk_load_tile(const R *src, uint64_t base, const Stage<R, E> &tc,
                                               typename Vec2<R>::type *tile, uint64_t *bar) {
  using C2 = typename Vec2<R>::type;
  const uint32_t nch = 1u << (tc.T - tc.C);
  const uint32_t bytes = (uint32_t)sizeof(C2) << tc.C;
  const C2 *g = reinterpret_cast<const C2 *>(src);
  if (threadIdx.x == 0) mbar_expect_tx(bar, bytes * nch);
  for (uint32_t h = threadIdx.x; h < nch; h += NT) bulk_g2s(tile + (h << tc.C), g + (base ^ tc.off[h]), bytes, bar);
}

// Write tile `base` back; the caller has fenced its shared-memory writes and synced.
template <typename R, typename E>
__device__ __forceinline__ void bulk_store_tile(R *dst, uint64_t base, const Stage<R, E> &tc,
                                                const typename Vec2<R>::type *tile) {
  using C2 = typename Vec2<R>::type;
  const uint32_t nch = 1u << (tc.T - tc.C);
  const uint32_t bytes = (uint32_t)sizeof(C2) << tc.C;
  C2 *g = reinterpret_cast<C2 *>(dst);
  for (uint32_t h = threadIdx.x; h < nch; h += NT) bulk_s2g(g + (base ^ tc.off[h]), tile + (h << tc.C), bytes);
  bulk_commit();
}

// ------------------------------------------------------------------ complex helpers

template <typename C2, typename R>
__device__ __forceinline__ void rot_real(C2 &a, C2 &b, R c, R s) {   // [[c,-s],[s,c]]
  const C2 x = a, y = b;
  a = C2{c * x.x - s * y.x, c * x.y - s * y.y};
  b = C2{s * x.x + c * y.x, s * x.y + c * y.y};
}
template <typename C2, typename R>
__device__ __forceinline__ void rot_xrot(C2 &a, C2 &b, R c, R s) {   // c - i s X
  const C2 x = a, y = b;
  a = C2{c * x.x + s * y.y, c * x.y - s * y.x};
  b = C2{c * y.x + s * x.y, c * y.y - s * x.x};
}
template <typename C2, typename R>
__device__ __forceinline__ void phase(C2 &a, R c, R s) {               // (c - i s) a
  const C2 x = a;
  a = C2{c * x.x + s * x.y, c * x.y - s * x.x};
}

// Packed FP32 pairs: one instruction updates (re, im) of an amplitude.
__device__ __forceinline__ unsigned long long f2_pack(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// [[c, -s], [s, c]] on (a, b) with e = (c, c, s, s).
__device__ __forceinline__ void rot_real(float2 &a, float2 &b, float4 e) {
  const unsigned long long A = f2_pack(a.x, a.y), B = f2_pack(b.x, b.y);
  const unsigned long long C = f2_pack(e.x, e.y), S = f2_pack(e.z, e.w);
  const unsigned long long na = f2_sub(f2_mul(C, A), f2_mul(S, B));
  const unsigned long long nb = f2_fma(S, A, f2_mul(C, B));
  a = f2_unpack(na);
  b = f2_unpack(nb);
}
template <typename C2, typename E>
__device__ __forceinline__ void rot_real(C2 &a, C2 &b, E e) {
  rot_real(a, b, lut_cos(e), lut_sin(e));
}

// ------------------------------------------------------------------ init

template <typename R>
__global__ void k_init_hf(R *psi, uint64_t n_amps, uint64_t hf) {
  using V = typename Vec16<R>::type;
  V *g = reinterpret_cast<V *>(psi);
  const uint64_t nv = (n_amps + Vec16<R>::amps - 1) / Vec16<R>::amps;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < nv;
       v += (uint64_t)gridDim.x * blockDim.x) {
    R e[4] = {0, 0, 0, 0};
    if (v == hf / Vec16<R>::amps) e[2 * (hf % Vec16<R>::amps)] = (R)1;
    V out;
    if constexpr (Vec16<R>::amps == 2) out = make_float4(e[0], e[1], e[2], e[3]);
    else out = make_double2(e[0], e[1]);
    g[v] = out;
  }
}

// ------------------------------------------------------------------ register blocks

// Cosets per thread of a D-dimensional block in a 2^TT tile (TT >= D + 8).
template <int TT, int D> struct BlockShape {
  static constexpr int J = (1 << (TT - D)) / NT;
  static constexpr int N = 1 << D;
};

// Rotate the pairs (c, c ^ A) of a coset held in registers.  REAL: the pair
// update [[c, -s], [s, c]]; otherwise c - i s X.
template <typename R, int D, int A, bool REAL, typename E>
__device__ __forceinline__ void coset_pairs(typename Vec2<R>::type (&v)[1 << D], const uint32_t (&bw)[4],
                                            const E *L, uint32_t cb) {
  constexpr int HB = 31 - __builtin_clz(A);
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    if ((c >> HB) & 1) continue;
    const uint32_t code = (bw[c >> 2] >> (8 * (c & 3))) & 0xffu;   // combo c's code byte
    const E cs = L[cb ^ code];
    if (REAL) rot_real(v[c], v[c ^ A], cs);
    else rot_xrot(v[c], v[c ^ A], lut_cos(cs), lut_sin(cs));
  }
}

// One jump on the pair offset a (1 .. 2^D - 1) into the unrolled pair loop.
template <typename R, int D, bool REAL, typename E>
__device__ __forceinline__ void coset_pairs_sw(int a, typename Vec2<R>::type (&v)[1 << D],
                                               const uint32_t (&bw)[4], const E *L, uint32_t cb) {
  switch (a) {
#define Q2_PC(X) \
  case X:        \
    if constexpr (X < (1 << D)) coset_pairs<R, D, X, REAL, E>(v, bw, L, cb); \
    break;
    Q2_PC(1) Q2_PC(2) Q2_PC(3) Q2_PC(4) Q2_PC(5) Q2_PC(6) Q2_PC(7) Q2_PC(8)
    Q2_PC(9) Q2_PC(10) Q2_PC(11) Q2_PC(12) Q2_PC(13) Q2_PC(14) Q2_PC(15)
#undef Q2_PC
    default: break;
  }
}

__host__ __device__ constexpr int log2_int(unsigned v) { return v <= 1 ? 0 : 1 + log2_int(v >> 1); }

// Byte offsets of the 2^D combos of a coset, built by one XOR each:
// off(c) = off(c without its top bit) ^ W[top bit].
template <int D>
__device__ __forceinline__ uint32_t combo_off(uint32_t o0, const uint32_t (&W)[D], int c) {
  uint32_t o = o0;
#pragma unroll
  for (int i = 0; i < D; ++i)
    if ((c >> i) & 1) o ^= W[i];
  return o;
}

// Byte offsets (from the start of shared memory) of a canonical group's LUT
// entries for the combos of one coset: the group's table starts at a
// multiple of 2^r entries, so entry (cb ^ code) sits at goff | (cb ^ code) << ES
// and XOR walks from one combo's entry to the next.
template <int D, int ES>
__device__ __forceinline__ void group_gens(const GroupDesc &g, int skip, uint32_t (&G)[D]) {
  const uint4 b4 = *reinterpret_cast<const uint4 *>(g.bccode);
  const uint32_t bw[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const int c = 1 << i;
    G[i] = i == skip ? 0u : (((bw[c >> 2] >> (8 * (c & 3))) & 0xffu) << ES);
  }
}

// Groups K..D-1 of a canonical block: group k pairs along basis bit k and is REAL.
template <typename R, int D, int K, typename E>
__device__ __forceinline__ void sweep_canon(typename Vec2<R>::type (&v)[1 << D], const Stage<R, E> &s, int gb,
                                            uint32_t lane, uint32_t warp, int j) {
  if constexpr (K < D) {
    constexpr int ES = log2_int(sizeof(E));
    const GroupDesc &g = s.gs[gb + K];
    const uint32_t cb = s.tcode[gb + K] ^ g.blane[lane] ^ g.bwarp[warp] ^ g.bjcode[j];
    const uint32_t goff = (uint32_t)(reinterpret_cast<const unsigned char *>(s.lut + g.lut) - s.base);
    const uint32_t lp = goff | (cb << ES);
    uint32_t G[D];
    group_gens<D, ES>(g, K, G);
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
      if ((c >> K) & 1) continue;
      const E cs = *reinterpret_cast<const E *>(s.base + combo_off<D>(lp, G, c));
      rot_real(v[c], v[c | (1 << K)], cs);
    }
    sweep_canon<R, D, K + 1, E>(v, s, gb, lane, warp, j);
  }
}

// One register block of the sweep.  J cosets per thread (GUARD: at most one).
template <typename R, int D, int J, bool GUARD>
__device__ __forceinline__ void sweep_block(typename Vec2<R>::type *tile, const BlockDesc &B,
                                            const Stage<R, typename SweepLut<R>::E> &s) {
  using C2 = typename Vec2<R>::type;
  using E = typename SweepLut<R>::E;
  constexpr int N = 1 << D;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (GUARD && tid >= (s.amps >> D)) return;
  uint32_t bt = tid;
#pragma unroll
  for (int i = 0; i < D; ++i) bt = insert_zero(bt, B.piv[i]);
  const int gb = B.g_begin, ge = B.g_end;
  constexpr int CS = log2_int(sizeof(C2));
  unsigned char *tb = reinterpret_cast<unsigned char *>(tile);
  uint32_t W[D];
#pragma unroll
  for (int i = 0; i < D; ++i) W[i] = (uint32_t)B.comb[1 << i] << CS;
#pragma unroll 1
  for (int j = 0; j < J; ++j) {
    const uint32_t o0 = (bt ^ B.uj[j]) << CS;
    C2 v[N];
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = *reinterpret_cast<const C2 *>(tb + combo_off<D>(o0, W, c));
    int g0 = gb;
    if (!GUARD && B.canon == D) {
      sweep_canon<R, D, 0, E>(v, s, gb, lane, warp, j);
      g0 = gb + D;
    }
#pragma unroll 1
    for (int gi = g0; gi < ge; ++gi) {
      const GroupDesc &g = s.gs[gi];
      const uint32_t cb = s.tcode[gi] ^ g.blane[lane] ^ g.bwarp[warp] ^ g.bjcode[j];
      const E *L = s.lut + g.lut;
      const uint4 b4 = *reinterpret_cast<const uint4 *>(g.bccode);   // all combo codes in one load
      const uint32_t bw[4] = {b4.x, b4.y, b4.z, b4.w};
      const int kind = g.kind;
      if (kind == KIND_REAL) {
        coset_pairs_sw<R, D, true, E>(g.a, v, bw, L, cb);
      } else if (kind == KIND_DIAG) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
          const E cs = L[cb ^ g.bccode[c]];
          phase(v[c], lut_cos(cs), lut_sin(cs));
        }
      } else {
        coset_pairs_sw<R, D, false, E>(g.a, v, bw, L, cb);
      }
    }
#pragma unroll
    for (int c = 0; c < N; ++c) *reinterpret_cast<C2 *>(tb + combo_off<D>(o0, W, c)) = v[c];
  }
}

template <typename R, int TT, bool GUARD>
__device__ __forceinline__ void sweep_block_any(typename Vec2<R>::type *tile, const BlockDesc &B,
                                                const Stage<R, typename SweepLut<R>::E> &s) {
  if constexpr (GUARD) {
    sweep_block<R, 1, 1, true>(tile, B, s);
  } else {
    switch (B.d) {
      case 1: sweep_block<R, 1, BlockShape<TT, 1>::J, false>(tile, B, s); break;
      case 2:
        if constexpr (TT >= 10) sweep_block<R, 2, BlockShape<TT, 2>::J, false>(tile, B, s);
        break;
      case 3:
        if constexpr (TT >= 11) sweep_block<R, 3, BlockShape<TT, 3>::J, false>(tile, B, s);
        break;
      case 4:
        if constexpr (TT >= 12) sweep_block<R, 4, BlockShape<TT, 4>::J, false>(tile, B, s);
        break;
    }
  }
}

// Per-thread asynchronous tile copies (the two fast kernels).  A bulk copy is
// one instruction per chunk whose operands differ from lane to lane, and ncu
// counts about 2,000 instructions per CTA for the 256 chunk copies of a 2^12
// tile each way; 16-byte cp.async copies, consecutive threads on consecutive
// pieces, take 8 per thread and a hardware dependency wait (no poll).  Stores
// go the plain way (store_tile), from shared memory through registers.
template <typename R, typename E>
__device__ __forceinline__ void async_load_tile(const R *src, uint64_t base, const Stage<R, E> &tc,
                                                typename Vec2<R>::type *tile) {
  using V = typename Vec16<R>::type;
  constexpr int A = Vec16<R>::amps;
  const uint32_t nv = tc.amps / A;
  const uint32_t cm = (1u << tc.C) - 1u;
  const V *g = reinterpret_cast<const V *>(src);
  const uint32_t sb = smem_u32(tile);
#pragma unroll 4
  for (uint32_t v = threadIdx.x; v < nv; v += NT) {
    const uint32_t l = v * A;
    const uint64_t i = (base ^ tc.off[l >> tc.C]) | (l & cm);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sb + v * 16u), "l"((const void *)(g + i / A))
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// Wait for this thread's asynchronous copies; the caller then syncs the CTA.
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Write tile `base` back and start the copy of tile `next` into the same shared
// memory: each thread moves the 16-byte pieces it owns in both copies (pieces
// tid, tid + NT, ...), so once a piece is in registers and stored, the thread
// may refill it without waiting for the CTA.  Eight pieces per batch.
template <int TT, bool STREAM, typename E>
__device__ __forceinline__ void store_load_tile(float *psi, uint64_t base, uint64_t next, const Stage<float, E> &tc,
                                                float2 *tile) {
  using V = typename Vec16<float>::type;
  constexpr int A = Vec16<float>::amps;
  constexpr int PER = (1 << TT) / A / NT;   // pieces per thread
  constexpr int BATCH = PER < 8 ? PER : 8;
  const uint32_t cm = (1u << tc.C) - 1u;
  V *g = reinterpret_cast<V *>(psi);
  const V *tv = reinterpret_cast<const V *>(tile);
  const uint32_t sb = smem_u32(tile);
#pragma unroll
  for (int k0 = 0; k0 < PER; k0 += BATCH) {
    V buf[BATCH];
#pragma unroll
    for (int k = 0; k < BATCH; ++k) buf[k] = tv[(k0 + k) * NT + threadIdx.x];
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const uint32_t v = (k0 + k) * NT + threadIdx.x, l = v * A;
      st16<V, STREAM>(g + ((base ^ tc.off[l >> tc.C]) | (l & cm)) / A, buf[k]);
    }
#pragma unroll
    for (int k = 0; k < BATCH; ++k) {
      const uint32_t v = (k0 + k) * NT + threadIdx.x, l = v * A;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sb + v * 16u),
                   "l"((const void *)(g + ((next ^ tc.off[l >> tc.C]) | (l & cm)) / A))
                   : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// ------------------------------------------------------------------ canonical 4-dimensional sweep blocks
//
// Fast path for passes whose register blocks are all canonical and 4-dimensional
// with exactly four groups (group k pairs combos c and c | 1 << k and is REAL):
// the shape of every block of a UCCSD double-excitation sweep.  Everything in a
// group's addressing that does not depend on the tile is computed once per CTA
// and pass:
//   thr[g][tid]  code of the thread's coset base, blane[lane] ^ bwarp[warp];
//   C4Group[g]   byte offset of the group's LUT in shared memory and its four
//                pair generators (bccode[1 << i] << 4, one per block dimension);
//   btab[b][tid] byte offset of the thread's coset base in the tile.
// Per tile and group only the tile code is added.  Amplitudes are kept as packed
// 64-bit (re, im) registers for the f32x2 instructions, and the combos of a coset
// and the LUT entries of a group are walked in Gray-code order, one XOR per step.
// Tiles come in by per-thread async copies and go out by plain streaming stores.

constexpr int C4_MAX_GROUPS = 16;   // groups of a pass on this path (4 blocks)

struct alignas(16) C4Group {
  uint32_t lutoff;   // shared-window address of the group's LUT (a multiple of its size)
  uint32_t g01;      // pair generators of block dimensions 0 and 1 (u16 each, already << 4)
  uint32_t g23;      // ... of dimensions 2 and 3
  uint32_t pad;
};

__host__ __device__ inline size_t c4_extra_bytes(int ng, int nb) {
  return align16((size_t)ng * NT) + sizeof(C4Group) * (size_t)ng + align16(sizeof(uint16_t) * NT * (size_t)nb);
}

__device__ __forceinline__ uint32_t c4_gen(const C4Group &g, int i) {
  return i == 0 ? (g.g01 & 0xffffu) : i == 1 ? (g.g01 >> 16) : i == 2 ? (g.g23 & 0xffffu) : (g.g23 >> 16);
}

// Rotation [[c, -s], [s, c]] of a packed complex pair with C = (c, c), S = (s, s).
__device__ __forceinline__ void rot_real_packed(unsigned long long &a, unsigned long long &b, unsigned long long C,
                                                unsigned long long S) {
  const unsigned long long na = f2_sub(f2_mul(C, a), f2_mul(S, b));
  const unsigned long long nb = f2_fma(S, a, f2_mul(C, b));
  a = na;
  b = nb;
}

// Index of the lowest set bit of v (1 <= v < 16), usable in device constant expressions.
__host__ __device__ constexpr int ctz_c(int v) { return (v & 1) ? 0 : (v & 2) ? 1 : (v & 4) ? 2 : 3; }
// Gray code: step t visits t ^ (t >> 1); the bit flipped after step t is ctz(t + 1).
__host__ __device__ constexpr int gray_flip3(int t) { return ctz_c(t + 1); }
__host__ __device__ constexpr int gray3(int t) { return t ^ (t >> 1); }
__host__ __device__ constexpr int gray_flip4(int t) { return ctz_c(t + 1); }
__host__ __device__ constexpr int gray4(int t) { return t ^ (t >> 1); }

// Combo c of group K's pair p (p = 0..7): the three bits other than K carry p.
template <int K> __host__ __device__ constexpr int c4_combo(int p) {
  return K == 0 ? (p << 1) : K == 1 ? ((p & 1) | ((p & 6) << 1)) : K == 2 ? ((p & 3) | ((p & 4) << 1)) : p;
}
// Block dimension of the i-th bit of a pair index of group K.
template <int K> __host__ __device__ constexpr int c4_dim(int i) { return i < K ? i : i + 1; }

// Group K of a canonical block on one coset held in v[16].
template <int K>
__device__ __forceinline__ void c4_group(unsigned long long (&v)[16], uint32_t A, const C4Group &cg) {
  const uint32_t G0 = c4_gen(cg, c4_dim<K>(0)), G1 = c4_gen(cg, c4_dim<K>(1)), G2 = c4_gen(cg, c4_dim<K>(2));
  uint32_t addr = A;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    constexpr int dummy = 0;
    (void)dummy;
    const int p = gray3(t);
    const int c = c4_combo<K>(p);
    const ulonglong2 e = lds_b128(addr);
    rot_real_packed(v[c], v[c | (1 << K)], e.x, e.y);
    if (t < 7) {
      const int f = gray_flip3(t);
      addr ^= f == 0 ? G0 : f == 1 ? G1 : G2;
    }
  }
}

// One canonical 4-dimensional block: J cosets per thread (16 amplitudes each).
template <int J>
__device__ __forceinline__ void sweep_block_c4(float2 *tile, const BlockDesc &B, int b, const Stage<float, float4> &s,
                                               const unsigned char *thr, const C4Group *cgs, const uint16_t *btab) {
  const uint32_t tid = threadIdx.x;
  const uint32_t tb = smem_u32(tile);   // shared-window address of the tile
  const uint32_t W0 = (uint32_t)B.comb[1] << 3, W1 = (uint32_t)B.comb[2] << 3, W2 = (uint32_t)B.comb[4] << 3,
                 W3 = (uint32_t)B.comb[8] << 3;
  const int gb = B.g_begin;
  const uint32_t bt = btab[b * NT + tid];
#pragma unroll 1
  for (int j = 0; j < J; ++j) {
    unsigned long long v[16];
    uint32_t o = (bt ^ B.uj[j]) << 3;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      v[gray4(t)] = lds_b64(tb + o);
      if (t < 15) {
        const int f = gray_flip4(t);
        o ^= f == 0 ? W0 : f == 1 ? W1 : f == 2 ? W2 : W3;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int g = gb + k;
      const GroupDesc &gd = s.gs[g];
      const uint32_t cb = s.tcode[g] ^ thr[g * NT + tid] ^ gd.bjcode[j];
      const C4Group cg = cgs[g];
      const uint32_t A = cg.lutoff | (cb << 4);
      if (k == 0) c4_group<0>(v, A, cg);
      else if (k == 1) c4_group<1>(v, A, cg);
      else if (k == 2) c4_group<2>(v, A, cg);
      else c4_group<3>(v, A, cg);
    }
    // o is now the address of combo gray4(15) = 8; walk back in the same order to store
#pragma unroll
    for (int t = 15; t >= 0; --t) {
      sts_b64(tb + o, v[gray4(t)]);
      if (t > 0) {
        const int f = gray_flip4(t - 1);
        o ^= f == 0 ? W0 : f == 1 ? W1 : f == 2 ? W2 : W3;
      }
    }
  }
}

// Per-CTA tables of the canonical path (after stage_pass; the caller syncs).
__device__ __forceinline__ void stage_c4(const Stage<float, float4> &s, const PassDesc &pd, unsigned char *extra,
                                         unsigned char **thr, C4Group **cgs, uint16_t **btab) {
  const int ng = pd.g_end - pd.g_begin, nb = pd.b_end - pd.b_begin;
  unsigned char *t = extra;
  C4Group *c = reinterpret_cast<C4Group *>(t + align16((size_t)ng * NT));
  uint16_t *bt = reinterpret_cast<uint16_t *>(c + ng);
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int g = 0; g < ng; ++g) t[g * NT + tid] = s.gs[g].blane[lane] ^ s.gs[g].bwarp[warp];
  if ((int)tid < ng) {
    const GroupDesc &d = s.gs[tid];
    C4Group r;
    r.lutoff = smem_u32(s.lut + d.lut);   // absolute shared address, aligned to the group's table size
    r.g01 = ((uint32_t)d.bccode[1] << 4) | ((uint32_t)d.bccode[2] << 20);
    r.g23 = ((uint32_t)d.bccode[4] << 4) | ((uint32_t)d.bccode[8] << 20);
    r.pad = 0;
    c[tid] = r;
  }
  for (int b = 0; b < nb; ++b) {
    uint32_t v = tid;
#pragma unroll
    for (int i = 0; i < 4; ++i) v = insert_zero(v, s.bs[b].piv[i]);
    bt[b * NT + tid] = (uint16_t)v;
  }
  *thr = t;
  *cgs = c;
  *btab = bt;
}

// ------------------------------------------------------------------ rotation sweep

template <typename R, bool STREAM, int TT, bool GUARD>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 4 : 3)
    k_sweep(R *psi, int n, PassDesc pd, const GroupDesc *groups, const BlockDesc *blocks,
            const typename Vec2<R>::type *lut, unsigned *fault) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  using E = typename SweepLut<R>::E;
  const SmemLayout L = smem_layout(sizeof(C2), pd, 1, 0, sizeof(E), sizeof(E) << R_MAX_ROT);
  const Stage<R, E> st = stage_pass<R, E>(smem, pd, L, groups, blocks, lut);
  C2 *tile = reinterpret_cast<C2 *>(smem + L.tiles);
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const int ng = pd.g_end - pd.g_begin, nb = pd.b_end - pd.b_begin;
  if constexpr (GUARD) {   // tiles below 2^9 amplitudes: plain loads and stores
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const uint64_t base = tile_base(t, pd.umask);
      load_tile<R, STREAM>(psi, base, st, reinterpret_cast<V *>(tile));
      tile_codes(st, ng, t);
      __syncthreads();
      for (int b = 0; b < nb; ++b) {
        sweep_block_any<R, TT, GUARD>(tile, st.bs[b], st);
        __syncthreads();
      }
      store_tile<R, STREAM>(psi, base, st, reinterpret_cast<const V *>(tile));
      __syncthreads();
    }
  } else {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t parity = 0;
    TileWalk tw(blockIdx.x, gridDim.x, pd.umask);
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, tw.next()) {
      const uint64_t base = tw.base;
      bulk_load_tile(psi, base, st, tile, &bar);
      tile_codes(st, ng, t);
      const bool ok = mbar_wait(&bar, parity, fault);
      parity ^= 1u;
      if (__syncthreads_or(!ok)) {
        mbar_wait(&bar, parity ^ 1u, fault);   // a second bounded wait for the copies in flight
        break;
      }
      for (int b = 0; b < nb; ++b) {
        sweep_block_any<R, TT, GUARD>(tile, st.bs[b], st);
        __syncthreads();
      }
      fence_proxy_async();   // this thread's tile writes -> visible to the bulk store
      __syncthreads();
      bulk_store_tile(psi, base, st, tile);
      bulk_wait_read();      // the tile may be overwritten once every store has read it
      __syncthreads();
    }
    bulk_wait_all();
  }
}

// The pass loop of the canonical 4-dimensional fast path (complex64, 12- and
// 13-qubit tiles), as a kernel of its own so that its registers are allocated
// for this path alone.  (A variant with two tile buffers per CTA, at three CTAs
// per SM, measured slower than one buffer at four CTAs per SM.)
template <bool STREAM, int TT>
__global__ void __launch_bounds__(NT, 4)
    k_sweep_c4(float *psi, int n, PassDesc pd, const GroupDesc *groups, const BlockDesc *blocks, const float2 *lut) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ng = pd.g_end - pd.g_begin, nb = pd.b_end - pd.b_begin;
  constexpr size_t LA = sizeof(float4) << R_MAX_ROT;
  const SmemLayout L = smem_layout(sizeof(float2), pd, 1, c4_extra_bytes(ng, nb), sizeof(float4), LA, LA);
  const Stage<float, float4> st =
      stage_pass<float, float4>(smem, pd, L, groups, blocks, lut, abs_align_shift(smem, L.lut, LA));
  float2 *tile = reinterpret_cast<float2 *>(smem + L.tiles);
  __syncthreads();
  unsigned char *thr;
  C4Group *cgs;
  uint16_t *btab;
  stage_c4(st, pd, smem + L.extra, &thr, &cgs, &btab);
  __syncthreads();
  using V = typename Vec16<float>::type;
  const uint64_t ntiles = 1ull << (n - pd.T);
  TileWalk tw(blockIdx.x, gridDim.x, pd.umask);
  if (blockIdx.x < ntiles) async_load_tile(psi, tw.base, st, tile);
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tw.base;
    tw.next();   // tw.base: the next tile of this CTA
    tile_codes(st, ng, t);
    cp_async_wait_all();
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
      sweep_block_c4<BlockShape<TT, 4>::J>(tile, st.bs[b], b, st, thr, cgs, btab);
      if (b + 1 < nb) __syncthreads();
    }
    __syncthreads();   // the tile is final and every group's tile code has been read
    if (t + gridDim.x < ntiles) store_load_tile<TT, STREAM>(psi, base, tw.base, st, tile);
    else store_tile<float, STREAM>(psi, base, st, reinterpret_cast<const V *>(tile));
  }
}

// ------------------------------------------------------------------ reductions

// Compensated (Kahan) accumulation in the state precision.
template <typename R> struct Kahan {
  R s = 0, c = 0;
  __device__ __forceinline__ void add(R v) {
    const R y = v - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Sum a double over the CTA; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *scratch) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += scratch[w];
  return s;
}

// ------------------------------------------------------------------ expectation

// sum over the pairs (c, c ^ A) of a coset of R Re w + Q Im w, w = conj(v_c) v_{c^A},
// (R, Q) = L[cb ^ code(c)]; the caller doubles it (each pair counts i<j and j>i).
// QZERO: the group's Q vanishes at every code (real pair coefficients).
template <typename R, int D, int A, bool QZERO>
__device__ __forceinline__ R coset_expect(const typename Vec2<R>::type (&v)[1 << D], uint2 b2,
                                          const typename Vec2<R>::type *L, uint32_t cb) {
  constexpr int HB = 31 - __builtin_clz(A);
  const uint32_t bw[2] = {b2.x, b2.y};
  R s = 0;
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    if ((c >> HB) & 1) continue;
    const uint32_t idx = cb ^ ((bw[c >> 2] >> (8 * (c & 3))) & 0xffu);
    const auto a = v[c], b = v[c ^ A];
    if constexpr (QZERO) {
      s += L[idx].x * (a.x * b.x + a.y * b.y);
    } else {
      const auto rq = L[idx];
      s += rq.x * (a.x * b.x + a.y * b.y) + rq.y * (a.x * b.y - a.y * b.x);
    }
  }
  return s;
}

// e[j] += 2 * coset_expect(v[j]) for every coset of a chunk; one jump on a.
template <typename R, int D, int JC, bool QZERO>
__device__ __forceinline__ void chunk_expect(int a, const typename Vec2<R>::type (&v)[JC][1 << D], R (&e)[JC],
                                             uint2 b2, const typename Vec2<R>::type *L, uint32_t cb,
                                             const uint8_t *bjcode) {
  switch (a) {
#define Q2_EC(X)                                                              \
  case X:                                                                     \
    if constexpr (X < (1 << D)) {                                             \
      _Pragma("unroll") for (int j = 0; j < JC; ++j)                          \
        e[j] += 2 * coset_expect<R, D, X, QZERO>(v[j], b2, L, cb ^ bjcode[j]); \
    }                                                                         \
    break;
    Q2_EC(1) Q2_EC(2) Q2_EC(3) Q2_EC(4) Q2_EC(5) Q2_EC(6) Q2_EC(7)
#undef Q2_EC
    default: break;
  }
}

// Groups K..D-1 of a canonical block: group k pairs along basis bit k, Q = 0.
template <typename R, int D, int JC, int K>
__device__ __forceinline__ void expect_canon(const typename Vec2<R>::type (&v)[JC][1 << D], R (&e)[JC],
                                             const Stage<R> &s, int gb, uint32_t lane, uint32_t warp, int j0) {
  if constexpr (K < D) {
    using C2 = typename Vec2<R>::type;
    constexpr int ES = log2_int(sizeof(C2));
    const GroupDesc &g = s.gs[gb + K];
    const uint32_t cb = s.tcode[gb + K] ^ g.blane[lane] ^ g.bwarp[warp];
    const uint32_t goff = (uint32_t)(reinterpret_cast<const unsigned char *>(s.lut + g.lut) - s.base);
    uint32_t G[D];
    group_gens<D, ES>(g, K, G);
#pragma unroll
    for (int j = 0; j < JC; ++j) {
      const uint32_t lp = goff | ((cb ^ g.bjcode[j0 + j]) << ES);
      R t = 0;
#pragma unroll
      for (int c = 0; c < (1 << D); ++c) {
        if ((c >> K) & 1) continue;
        const R r = *reinterpret_cast<const R *>(s.base + combo_off<D>(lp, G, c));
        const C2 a = v[j][c], b = v[j][c | (1 << K)];
        t += r * (a.x * b.x + a.y * b.y);
      }
      e[j] += 2 * t;
    }
    expect_canon<R, D, JC, K + 1>(v, e, s, gb, lane, warp, j0);
  }
}

// One register block of the expectation.  The thread's J cosets are taken in
// chunks of JC (JC * 2^D amplitudes in registers); for each chunk it walks the
// block's groups once.  Each coset's contribution is summed over the groups in
// the state precision and enters the compensated accumulator once per block.
template <typename R, int D, int J, bool GUARD>
__device__ __forceinline__ void expect_block(const typename Vec2<R>::type *tile, const BlockDesc &B,
                                             const Stage<R> &s, Kahan<R> &acc) {
  using C2 = typename Vec2<R>::type;
  constexpr int N = 1 << D;
  constexpr int AMPS = 8;   // amplitudes a thread keeps in registers per chunk
  constexpr int JC = J < AMPS / N ? J : (AMPS / N > 0 ? AMPS / N : 1);
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (GUARD && tid >= (s.amps >> D)) return;
  uint32_t bt = tid;
#pragma unroll
  for (int i = 0; i < D; ++i) bt = insert_zero(bt, B.piv[i]);
  const int gb = B.g_begin, ge = B.g_end;
  constexpr int CS = log2_int(sizeof(C2));
  const unsigned char *tb = reinterpret_cast<const unsigned char *>(tile);
  uint32_t W[D];
#pragma unroll
  for (int i = 0; i < D; ++i) W[i] = (uint32_t)B.comb[1 << i] << CS;
#pragma unroll 1
  for (int j0 = 0; j0 < J; j0 += JC) {
    C2 v[JC][N];
#pragma unroll
    for (int j = 0; j < JC; ++j) {
      const uint32_t o0 = (bt ^ B.uj[j0 + j]) << CS;
#pragma unroll
      for (int c = 0; c < N; ++c) v[j][c] = *reinterpret_cast<const C2 *>(tb + combo_off<D>(o0, W, c));
    }
    R e[JC];
#pragma unroll
    for (int j = 0; j < JC; ++j) e[j] = 0;
    int g0 = gb;
    if (!GUARD && B.canon == D) {
      expect_canon<R, D, JC, 0>(v, e, s, gb, lane, warp, j0);
      g0 = gb + D;
    }
#pragma unroll 1
    for (int gi = g0; gi < ge; ++gi) {
      const GroupDesc &g = s.gs[gi];
      const uint32_t cb = s.tcode[gi] ^ g.blane[lane] ^ g.bwarp[warp];
      const C2 *L = s.lut + g.lut;
      if (g.kind == KIND_DIAG) {
#pragma unroll
        for (int j = 0; j < JC; ++j) {
          const uint32_t cj = cb ^ g.bjcode[j0 + j];
#pragma unroll
          for (int c = 0; c < N; ++c)
            e[j] += L[cj ^ g.bccode[c]].x * (v[j][c].x * v[j][c].x + v[j][c].y * v[j][c].y);
        }
      } else {
        const uint2 b2 = *reinterpret_cast<const uint2 *>(g.bccode);   // combo codes c < 8 in one load
        if (g.kind == KIND_REAL) chunk_expect<R, D, JC, true>(g.a, v, e, b2, L, cb, g.bjcode + j0);
        else chunk_expect<R, D, JC, false>(g.a, v, e, b2, L, cb, g.bjcode + j0);
      }
    }
#pragma unroll
    for (int j = 0; j < JC; ++j) acc.add(e[j]);
  }
}

template <typename R, int TT, bool GUARD>
__device__ __forceinline__ void expect_block_any(const typename Vec2<R>::type *tile, const BlockDesc &B,
                                                 const Stage<R> &s, Kahan<R> &acc) {
  if constexpr (GUARD) {
    expect_block<R, 1, 1, true>(tile, B, s, acc);
  } else {
    switch (B.d) {
      case 1: expect_block<R, 1, BlockShape<TT, 1>::J, false>(tile, B, s, acc); break;
      case 2:
        if constexpr (TT >= 10) expect_block<R, 2, BlockShape<TT, 2>::J, false>(tile, B, s, acc);
        break;
      case 3:
        if constexpr (TT >= 11) expect_block<R, 3, BlockShape<TT, 3>::J, false>(tile, B, s, acc);
        break;
    }
  }
}

template <typename R, bool STREAM, int TT, bool GUARD>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 2 : 1) k_expect(const R *psi, int n, PassDesc pd,
                                                  const GroupDesc *groups, const BlockDesc *blocks,
                                                  const typename Vec2<R>::type *lut, double *partial,
                                                  int first_pass, unsigned *fault) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(sizeof(C2), pd, 1, sizeof(double) * (NT / 32), sizeof(C2), sizeof(C2) << R_MAX);
  const Stage<R> st = stage_pass<R>(smem, pd, L, groups, blocks, lut);
  C2 *tile = reinterpret_cast<C2 *>(smem + L.tiles);
  double *red = reinterpret_cast<double *>(smem + L.extra);
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const int ng = pd.g_end - pd.g_begin, nb = pd.b_end - pd.b_begin;
  Kahan<R> acc_e, acc_n;
  __shared__ uint64_t bar;
  if (!GUARD && threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t parity = 0;
  TileWalk tw(blockIdx.x, gridDim.x, pd.umask);
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, tw.next()) {
    if constexpr (GUARD) {
      load_tile<R, STREAM>(psi, tw.base, st, reinterpret_cast<V *>(tile));
      tile_codes(st, ng, t);
      __syncthreads();
    } else {
      bulk_load_tile(psi, tw.base, st, tile, &bar);
      tile_codes(st, ng, t);
      const bool ok = mbar_wait(&bar, parity, fault);
      parity ^= 1u;
      if (__syncthreads_or(!ok)) {
        mbar_wait(&bar, parity ^ 1u, fault);   // a second bounded wait for the copies in flight
        break;
      }
    }
    if (first_pass) {
      R s = 0;
      for (uint32_t l = threadIdx.x; l < st.amps; l += NT) {
        const C2 a = tile[l];
        s += a.x * a.x + a.y * a.y;
      }
      acc_n.add(s);
    }
    for (int b = 0; b < nb; ++b) expect_block_any<R, TT, GUARD>(tile, st.bs[b], st, acc_e);
    __syncthreads();
  }
  const double e = block_sum(acc_e.value(), red);
  const double nn = block_sum(acc_n.value(), red);
  if (threadIdx.x == 0) {
    if (first_pass) {
      partial[2 * blockIdx.x] = e;
      partial[2 * blockIdx.x + 1] = nn;
    } else {
      partial[2 * blockIdx.x] += e;
    }
  }
}

// ------------------------------------------------------------------ expectation, lean path
//
// Passes whose groups are all REAL (real pair coefficients) or DIAG, in register
// blocks of at most 3 dimensions, on 12- or 13-qubit tiles (complex64): each
// thread holds all of its cosets of a block (2^TT / NT amplitudes, packed 64-bit
// (re, im) registers) and walks every group of the block once.  The staged LUT
// holds (R, R) for these groups, so one f32x2 multiply and one f32x2 fused
// multiply-add give a pair's R (x_i x_j, y_i y_j); each group's sum enters the
// compensated accumulator once.  Per group and pass the LUT byte offset and
// the pair generators (bccode[1 << i] << 3) are staged once per CTA; the
// combos of a coset and a group's LUT entries are walked in Gray-code order.
// Tiles come in by per-thread async copies; the next tile's copy is issued as
// soon as the last block of the current tile is in registers.

struct alignas(16) EGroup {
  uint32_t lutoff;   // shared-window address of the group's LUT (a multiple of its size)
  uint32_t g01;      // pair generators of block dimensions 0 and 1 (u16 each, already << 3)
  uint32_t g2;       // ... of dimension 2
  uint32_t kind_a;   // kind | (a << 8)
  uint32_t bj[2];    // coset codes bjcode[0..3] << 3 as u16 (cosets of 3-dimensional blocks)
  uint32_t pad[2];
};

__host__ __device__ inline size_t efast_extra_bytes(int ng) {
  return sizeof(double) * (NT / 32) + sizeof(EGroup) * (size_t)ng;
}

__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// XOR of coset j's code (<< 3) into a LUT address: from the staged record for J <= 4,
// from the group descriptor otherwise.
template <int J>
__device__ __forceinline__ uint32_t coset_code3(const EGroup &e, const uint8_t *bj, int j) {
  if constexpr (J <= 4) return (j & 1) ? (e.bj[j >> 1] >> 16) : (e.bj[j >> 1] & 0xffffu);
  else return (uint32_t)bj[j] << 3;
}

__device__ __forceinline__ uint32_t egen(const EGroup &g, int i) {
  return i == 0 ? (g.g01 & 0xffffu) : i == 1 ? (g.g01 >> 16) : g.g2;
}

__host__ __device__ constexpr int free_bit(int hb, int i) { return i < hb ? i : i + 1; }
__host__ __device__ constexpr int deposit_free(int hb, int p) { return (p & ((1 << hb) - 1)) | ((p >> hb) << (hb + 1)); }
__host__ __device__ constexpr int hbit(int x) { return x >= 4 ? 2 : x >= 2 ? 1 : 0; }

__device__ __forceinline__ float f2_lo_plus_hi(unsigned long long v) {
  const float2 f = f2_unpack(v);
  return f.x + f.y;
}

// Pairs (c, c ^ X) of one REAL group over the thread's J cosets: sum of R (x_c x_p + y_c y_p).
template <int D, int J, int X>
__device__ __forceinline__ float efast_pairs(const unsigned long long (&v)[J][1 << D], uint32_t A, const uint8_t *bj,
                                             const EGroup &e) {
  constexpr int HB = hbit(X);
  constexpr int P = 1 << (D - 1);
  uint32_t G[D > 1 ? D - 1 : 1];
#pragma unroll
  for (int i = 0; i < D - 1; ++i) G[i] = egen(e, free_bit(HB, i));
  unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};   // independent chains
#pragma unroll
  for (int j = 0; j < J; ++j) {
    uint32_t a = A ^ coset_code3<J>(e, bj, j);
#pragma unroll
    for (int t = 0; t < P; ++t) {
      const int p = t ^ (t >> 1);
      const int c = deposit_free(HB, p);
      const unsigned long long rr = lds_b64(a);
      unsigned long long &ak = acc[(j * P + t) & 3];
      ak = f2_fma(rr, f2_mul(v[j][c], v[j][c ^ X]), ak);
      if (t + 1 < P) a ^= G[ctz_c(t + 1)];
    }
  }
  return f2_lo_plus_hi(f2_add(f2_add(acc[0], acc[1]), f2_add(acc[2], acc[3])));
}

template <int D, int J>
__device__ __forceinline__ float efast_switch(int x, const unsigned long long (&v)[J][1 << D], uint32_t A,
                                              const uint8_t *bj, const EGroup &e) {
  switch (x) {
#define Q2_FC(X) \
  case X:        \
    if constexpr (X < (1 << D)) return efast_pairs<D, J, X>(v, A, bj, e); \
    break;
    Q2_FC(1) Q2_FC(2) Q2_FC(3) Q2_FC(4) Q2_FC(5) Q2_FC(6) Q2_FC(7)
#undef Q2_FC
    default: break;
  }
  return 0.f;
}

// Issues the next tile's copy into the tile buffer once every thread holds its
// amplitudes of the last block of a tile in registers (the tile is read only).
struct EPrefetch {
  bool now;           // this is the tile's last block
  bool has_next;      // there is a next tile for this CTA
  uint64_t next_base;
  const float *psi;
  float2 *tile;
};

template <int D, int J>
__device__ __forceinline__ void expect_block_fast(const float2 *tile, const BlockDesc &B, const Stage<float> &s,
                                                  const EGroup *egs, Kahan<float> &acc, bool norm, Kahan<float> &acc_n,
                                                  const EPrefetch &pf) {
  constexpr int N = 1 << D;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t bt = tid;
#pragma unroll
  for (int i = 0; i < D; ++i) bt = insert_zero(bt, B.piv[i]);
  uint32_t W[D];
#pragma unroll
  for (int i = 0; i < D; ++i) W[i] = (uint32_t)B.comb[1 << i] << 3;
  const uint32_t tb = smem_u32(tile);   // shared-window address of the tile
  unsigned long long v[J][N];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    uint32_t o = (bt ^ B.uj[j]) << 3;
#pragma unroll
    for (int t = 0; t < N; ++t) {
      v[j][t ^ (t >> 1)] = lds_b64(tb + o);
      if (t + 1 < N) o ^= W[ctz_c(t + 1)];
    }
  }
  if (pf.now) {
    __syncthreads();   // every thread's reads of the tile are done
    if (pf.has_next) async_load_tile(pf.psi, pf.next_base, s, pf.tile);
  }
  if (norm) {   // every amplitude of the tile is in exactly one coset of this block
    unsigned long long n2[2] = {0ull, 0ull};
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int c = 0; c < N; ++c) n2[c & 1] = f2_fma(v[j][c], v[j][c], n2[c & 1]);
    acc_n.add(f2_lo_plus_hi(n2[0]) + f2_lo_plus_hi(n2[1]));
  }
#pragma unroll 1
  for (int gi = B.g_begin; gi < B.g_end; ++gi) {
    const GroupDesc &g = s.gs[gi];
    const EGroup e = egs[gi];
    const uint32_t cb = s.tcode[gi] ^ g.blane[lane] ^ g.bwarp[warp];
    const uint32_t A = e.lutoff | (cb << 3);
    const int kind = (int)(e.kind_a & 0xffu);
    float sum;
    if (kind == KIND_DIAG) {
      unsigned long long a2[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
      for (int j = 0; j < J; ++j) {
        uint32_t a = A ^ coset_code3<J>(e, g.bjcode, j);
#pragma unroll
        for (int t = 0; t < N; ++t) {
          const int c = t ^ (t >> 1);
          const unsigned long long rr = lds_b64(a);
          unsigned long long &ak = a2[(j * N + t) & 3];
          ak = f2_fma(rr, f2_mul(v[j][c], v[j][c]), ak);
          if (t + 1 < N) a ^= egen(e, ctz_c(t + 1));
        }
      }
      sum = f2_lo_plus_hi(f2_add(f2_add(a2[0], a2[1]), f2_add(a2[2], a2[3])));
    } else {
      sum = 2.f * efast_switch<D, J>((int)(e.kind_a >> 8), v, A, g.bjcode, e);
    }
    acc.add(sum);
  }
}

template <int TT>
__device__ __forceinline__ void expect_block_fast_any(const float2 *tile, const BlockDesc &B, const Stage<float> &s,
                                                      const EGroup *egs, Kahan<float> &acc, bool norm,
                                                      Kahan<float> &acc_n, const EPrefetch &pf) {
  switch (B.d) {
    case 1: expect_block_fast<1, BlockShape<TT, 1>::J>(tile, B, s, egs, acc, norm, acc_n, pf); break;
    case 2: expect_block_fast<2, BlockShape<TT, 2>::J>(tile, B, s, egs, acc, norm, acc_n, pf); break;
    default: expect_block_fast<3, BlockShape<TT, 3>::J>(tile, B, s, egs, acc, norm, acc_n, pf); break;
  }
}

template <bool STREAM, int TT>
__global__ void __launch_bounds__(NT, 2) k_expect_fast(const float *psi, int n, PassDesc pd, const GroupDesc *groups,
                                                       const BlockDesc *blocks, const float2 *lut, double *partial,
                                                       int first_pass) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ng = pd.g_end - pd.g_begin, nb = pd.b_end - pd.b_begin;
  constexpr size_t LA = sizeof(float2) << R_MAX;
  const SmemLayout L = smem_layout(sizeof(float2), pd, 1, efast_extra_bytes(ng), sizeof(float2), LA, LA);
  const Stage<float> st = stage_pass<float>(smem, pd, L, groups, blocks, lut, abs_align_shift(smem, L.lut, LA));
  float2 *tile = reinterpret_cast<float2 *>(smem + L.tiles);
  double *red = reinterpret_cast<double *>(smem + L.extra);
  EGroup *egs = reinterpret_cast<EGroup *>(red + NT / 32);
  __syncthreads();
  if ((int)threadIdx.x < ng) {
    const GroupDesc &d = st.gs[threadIdx.x];
    EGroup r;
    r.lutoff = smem_u32(st.lut + d.lut);   // absolute shared address, aligned to the group's table size
    r.g01 = ((uint32_t)d.bccode[1] << 3) | ((uint32_t)d.bccode[2] << 19);
    r.g2 = (uint32_t)d.bccode[4] << 3;
    r.kind_a = (uint32_t)d.kind | ((uint32_t)d.a << 8);
    r.bj[0] = ((uint32_t)d.bjcode[0] << 3) | ((uint32_t)d.bjcode[1] << 19);
    r.bj[1] = ((uint32_t)d.bjcode[2] << 3) | ((uint32_t)d.bjcode[3] << 19);
    r.pad[0] = r.pad[1] = 0;
    egs[threadIdx.x] = r;
  }
  const uint64_t ntiles = 1ull << (n - pd.T);
  Kahan<float> acc_e, acc_n;
  __syncthreads();
  TileWalk tw(blockIdx.x, gridDim.x, pd.umask);
  if (blockIdx.x < ntiles) async_load_tile(psi, tw.base, st, tile);
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    tw.next();   // tw.base: the next tile of this CTA
    tile_codes(st, ng, t);
    cp_async_wait_all();
    __syncthreads();
    EPrefetch pf{false, t + gridDim.x < ntiles, tw.base, psi, tile};
    for (int b = 0; b < nb; ++b) {
      pf.now = b == nb - 1;
      expect_block_fast_any<TT>(tile, st.bs[b], st, egs, acc_e, first_pass && b == 0, acc_n, pf);
    }
    __syncthreads();   // the tile codes of this tile are read by the last block's groups
  }
  const double e = block_sum(acc_e.value(), red);
  const double nn = block_sum(acc_n.value(), red);
  if (threadIdx.x == 0) {
    if (first_pass) {
      partial[2 * blockIdx.x] = e;
      partial[2 * blockIdx.x + 1] = nn;
    } else {
      partial[2 * blockIdx.x] += e;
    }
  }
}

// partial: [nblocks][2] -> out[0] = sum of energies, out[1] = sum of norms (fixed order)
__global__ void k_reduce_pairs(const double *partial, int nblocks, double *out) {
  __shared__ double sh[2][NT];
  double e = 0.0, nn = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    e += partial[2 * b];
    nn += partial[2 * b + 1];
  }
  sh[0][threadIdx.x] = e;
  sh[1][threadIdx.x] = nn;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sh[0][0];
    out[1] = sh[1][0];
  }
}

// ------------------------------------------------------------------ pair enumeration

// Pairs (or diagonal amplitudes) per thread of one group in a 2^TT tile.
template <int TT, bool GUARD> struct PairShape {
  static constexpr int P = GUARD ? 1 : (1 << (TT - 1)) / NT;
};

// ------------------------------------------------------------------ H apply

template <typename R, bool STREAM, int TT, bool GUARD>
__global__ void __launch_bounds__(NT, 3) k_happly(const R *psi, R *lam, int n, PassDesc pd,
                                                  const GroupDesc *groups,
                                                  const typename Vec2<R>::type *lut, int first_pass) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  constexpr int P = PairShape<TT, GUARD>::P;
  extern __shared__ __align__(16) unsigned char smem[];
  PassDesc pq = pd;
  pq.b_begin = pq.b_end = 0;
  const SmemLayout L = smem_layout(sizeof(C2), pq, 2, 0);
  const Stage<R> st = stage_pass<R>(smem, pq, L, groups, nullptr, lut);
  C2 *tp = reinterpret_cast<C2 *>(smem + L.tiles);
  C2 *tl = tp + st.amps;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const int ng = pd.g_end - pd.g_begin;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(t, pd.umask);
    load_tile<R, STREAM>(psi, base, st, reinterpret_cast<V *>(tp));
    if (first_pass) {
      for (uint32_t l = tid; l < st.amps; l += NT) tl[l] = C2{0, 0};
    } else {
      load_tile<R, STREAM>(lam, base, st, reinterpret_cast<V *>(tl));
    }
    tile_codes(st, ng, t);
    __syncthreads();
    for (int k = 0; k < ng; ++k) {
      const GroupDesc &d = st.gs[k];
      const C2 *lt = st.lut + d.lut;
      const uint32_t code0 = st.tcode[k] ^ d.plane[lane] ^ d.pwarp[warp];
      if (d.kind == KIND_DIAG) {
#pragma unroll
        for (int j = 0; j < 2 * P; ++j) {
          const uint32_t l = tid + NT * j;
          if (GUARD && l >= st.amps) break;
          const R dv = lt[code0 ^ d.pjcode[j]].x;
          const C2 a = tp[l];
          C2 o = tl[l];
          o.x += dv * a.x;
          o.y += dv * a.y;
          tl[l] = o;
        }
      } else if (!GUARD || tid < (st.amps >> 1)) {
        const uint32_t li0 = insert_zero(tid, d.pivot);
        const uint32_t xl = d.xl;
        const bool qzero = d.kind == KIND_REAL;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const uint32_t li = li0 | d.pu[j], lj = li ^ xl;
          const C2 rq = lt[code0 ^ d.pjcode[j]];
          const C2 a = tp[li], b = tp[lj];
          C2 oi = tl[li], oj = tl[lj];
          // lam_i += (R - iQ) psi_j ; lam_j += (R + iQ) psi_i
          if (qzero) {
            oi.x += rq.x * b.x;
            oi.y += rq.x * b.y;
            oj.x += rq.x * a.x;
            oj.y += rq.x * a.y;
          } else {
            oi.x += rq.x * b.x + rq.y * b.y;
            oi.y += rq.x * b.y - rq.y * b.x;
            oj.x += rq.x * a.x - rq.y * a.y;
            oj.y += rq.x * a.y + rq.y * a.x;
          }
          tl[li] = oi;
          tl[lj] = oj;
        }
      }
      __syncthreads();
    }
    store_tile<R, STREAM>(lam, base, st, reinterpret_cast<const V *>(tl));
    __syncthreads();
  }
}

// ------------------------------------------------------------------ register-blocked H apply
//
// lambda += H_pass psi on the Hamiltonian plan's register blocks: a thread
// holds a chunk of psi cosets and the matching lambda amplitudes in
// registers and walks the block's groups once; lambda goes back to the tile
// after each block.  Tiles move by bulk copies; the first pass starts from
// lambda = 0 without reading it.

// u[c] += (R - iQ) v[c ^ A], u[c ^ A] += (R + iQ) v[c] over the pairs (c, c ^ A).
template <typename R, int D, int A, bool QZERO>
__device__ __forceinline__ void coset_happly(const typename Vec2<R>::type (&v)[1 << D],
                                             typename Vec2<R>::type (&u)[1 << D], const unsigned char *base,
                                             uint32_t lp, const uint32_t (&G)[D]) {
  using C2 = typename Vec2<R>::type;
  constexpr int HB = 31 - __builtin_clz(A);
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    if ((c >> HB) & 1) continue;
    const C2 rq = *reinterpret_cast<const C2 *>(base + combo_off<D>(lp, G, c));
    const C2 a = v[c], b = v[c ^ A];
    if (QZERO) {
      u[c].x += rq.x * b.x;
      u[c].y += rq.x * b.y;
      u[c ^ A].x += rq.x * a.x;
      u[c ^ A].y += rq.x * a.y;
    } else {
      u[c].x += rq.x * b.x + rq.y * b.y;
      u[c].y += rq.x * b.y - rq.y * b.x;
      u[c ^ A].x += rq.x * a.x - rq.y * a.y;
      u[c ^ A].y += rq.x * a.y + rq.y * a.x;
    }
  }
}

template <typename R, int D, bool QZERO>
__device__ __forceinline__ void coset_happly_sw(int a, const typename Vec2<R>::type (&v)[1 << D],
                                                typename Vec2<R>::type (&u)[1 << D], const unsigned char *base,
                                                uint32_t lp, const uint32_t (&G)[D]) {
  switch (a) {
#define Q2_HC(X) \
  case X:        \
    if constexpr (X < (1 << D)) coset_happly<R, D, X, QZERO>(v, u, base, lp, G); \
    break;
    Q2_HC(1) Q2_HC(2) Q2_HC(3) Q2_HC(4) Q2_HC(5) Q2_HC(6) Q2_HC(7)
#undef Q2_HC
    default: break;
  }
}

// Groups K..D-1 of a canonical Hamiltonian block: group k pairs along basis bit k, Q = 0.
template <typename R, int D, int JC, int K>
__device__ __forceinline__ void happly_canon(const typename Vec2<R>::type (&v)[JC][1 << D],
                                             typename Vec2<R>::type (&u)[JC][1 << D], const Stage<R> &s, int gb,
                                             uint32_t lane, uint32_t warp, int j0) {
  if constexpr (K < D) {
    using C2 = typename Vec2<R>::type;
    constexpr int ES = log2_int(sizeof(C2));
    const GroupDesc &g = s.gs[gb + K];
    const uint32_t cb = s.tcode[gb + K] ^ g.blane[lane] ^ g.bwarp[warp];
    const uint32_t goff = (uint32_t)(reinterpret_cast<const unsigned char *>(s.lut + g.lut) - s.base);
    uint32_t G[D];
    group_gens<D, ES>(g, K, G);
#pragma unroll
    for (int j = 0; j < JC; ++j)
      coset_happly<R, D, 1 << K, true>(v[j], u[j], s.base, goff | ((cb ^ g.bjcode[j0 + j]) << ES), G);
    happly_canon<R, D, JC, K + 1>(v, u, s, gb, lane, warp, j0);
  }
}

template <typename R, int D, int J>
__device__ __forceinline__ void happly_block(const typename Vec2<R>::type *tp, typename Vec2<R>::type *tl,
                                             const BlockDesc &B, const Stage<R> &s) {
  using C2 = typename Vec2<R>::type;
  constexpr int N = 1 << D;
  constexpr int AMPS = 8;
  constexpr int JC = J < AMPS / N ? J : (AMPS / N > 0 ? AMPS / N : 1);
  constexpr int CS = log2_int(sizeof(C2));
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t bt = tid;
#pragma unroll
  for (int i = 0; i < D; ++i) bt = insert_zero(bt, B.piv[i]);
  const int gb = B.g_begin, ge = B.g_end;
  const unsigned char *pbase = reinterpret_cast<const unsigned char *>(tp);
  unsigned char *lbase = reinterpret_cast<unsigned char *>(tl);
  uint32_t W[D];
#pragma unroll
  for (int i = 0; i < D; ++i) W[i] = (uint32_t)B.comb[1 << i] << CS;
#pragma unroll 1
  for (int j0 = 0; j0 < J; j0 += JC) {
    C2 v[JC][N], u[JC][N];
#pragma unroll
    for (int j = 0; j < JC; ++j) {
      const uint32_t o0 = (bt ^ B.uj[j0 + j]) << CS;
#pragma unroll
      for (int c = 0; c < N; ++c) {
        v[j][c] = *reinterpret_cast<const C2 *>(pbase + combo_off<D>(o0, W, c));
        u[j][c] = *reinterpret_cast<const C2 *>(lbase + combo_off<D>(o0, W, c));
      }
    }
    int g0 = gb;
    if (B.canon == D) {
      happly_canon<R, D, JC, 0>(v, u, s, gb, lane, warp, j0);
      g0 = gb + D;
    }
#pragma unroll 1
    for (int gi = g0; gi < ge; ++gi) {
      const GroupDesc &g = s.gs[gi];
      const uint32_t cb = s.tcode[gi] ^ g.blane[lane] ^ g.bwarp[warp];
      constexpr int ES = log2_int(sizeof(C2));
      const uint32_t goff = (uint32_t)(reinterpret_cast<const unsigned char *>(s.lut + g.lut) - s.base);
      uint32_t G[D];
      group_gens<D, ES>(g, -1, G);
      if (g.kind == KIND_DIAG) {
#pragma unroll
        for (int j = 0; j < JC; ++j) {
          const uint32_t lp = goff | ((cb ^ g.bjcode[j0 + j]) << ES);
#pragma unroll
          for (int c = 0; c < N; ++c) {
            const R dv = reinterpret_cast<const C2 *>(s.base + combo_off<D>(lp, G, c))->x;
            u[j][c].x += dv * v[j][c].x;
            u[j][c].y += dv * v[j][c].y;
          }
        }
      } else {
        const int a = g.a;
        const bool qz = g.kind == KIND_REAL;
#pragma unroll
        for (int j = 0; j < JC; ++j) {
          const uint32_t lp = goff | ((cb ^ g.bjcode[j0 + j]) << ES);
          if (qz) coset_happly_sw<R, D, true>(a, v[j], u[j], s.base, lp, G);
          else coset_happly_sw<R, D, false>(a, v[j], u[j], s.base, lp, G);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < JC; ++j) {
      const uint32_t o0 = (bt ^ B.uj[j0 + j]) << CS;
#pragma unroll
      for (int c = 0; c < N; ++c) *reinterpret_cast<C2 *>(lbase + combo_off<D>(o0, W, c)) = u[j][c];
    }
  }
}

template <typename R, int TT>
__device__ __forceinline__ void happly_block_any(const typename Vec2<R>::type *tp, typename Vec2<R>::type *tl,
                                                 const BlockDesc &B, const Stage<R> &s) {
  switch (B.d) {
    case 1: happly_block<R, 1, BlockShape<TT, 1>::J>(tp, tl, B, s); break;
    case 2:
      if constexpr (TT >= 10) happly_block<R, 2, BlockShape<TT, 2>::J>(tp, tl, B, s);
      break;
    case 3:
      if constexpr (TT >= 11) happly_block<R, 3, BlockShape<TT, 3>::J>(tp, tl, B, s);
      break;
  }
}

template <typename R, int TT>
__global__ void __launch_bounds__(NT, 2) k_happly_blk(const R *psi, R *lam, int n, PassDesc pd,
                                                      const GroupDesc *groups, const BlockDesc *blocks,
                                                      const typename Vec2<R>::type *lut, int first_pass) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(sizeof(C2), pd, 2, 0, sizeof(C2), sizeof(C2) << R_MAX);
  const Stage<R> st = stage_pass<R>(smem, pd, L, groups, blocks, lut);
  C2 *tp = reinterpret_cast<C2 *>(smem + L.tiles);
  C2 *tl = tp + st.amps;
  const int ng = pd.g_end - pd.g_begin, nb = pd.b_end - pd.b_begin;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  TileWalk tw(blockIdx.x, gridDim.x, pd.umask);
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, tw.next()) {
    const uint64_t base = tw.base;
    async_load_tile(psi, base, st, tp);
    if (!first_pass) async_load_tile(lam, base, st, tl);
    else
      for (uint32_t l = threadIdx.x; l < st.amps; l += NT) tl[l] = C2{0, 0};
    tile_codes(st, ng, t);
    cp_async_wait_all();
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
      happly_block_any<R, TT>(tp, tl, st.bs[b], st);
      __syncthreads();
    }
    store_tile<R, false>(lam, base, st, reinterpret_cast<const V *>(tl));
    __syncthreads();   // every thread has read its pieces before the next tiles land
  }
}

// Re<psi|lam> and <psi|psi>, per-CTA partials.
template <typename R>
__global__ void __launch_bounds__(NT) k_dot(const R *psi, const R *lam, uint64_t n_amps,
                                            double *partial) {
  using C2 = typename Vec2<R>::type;
  __shared__ double red[NT / 32];
  const C2 *p = reinterpret_cast<const C2 *>(psi);
  const C2 *q = reinterpret_cast<const C2 *>(lam);
  Kahan<R> ae, an;
  const uint64_t stride = (uint64_t)gridDim.x * NT;
  for (uint64_t i0 = blockIdx.x * (uint64_t)NT + threadIdx.x; i0 < n_amps; i0 += 8 * stride) {
    R se = 0, sn = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint64_t i = i0 + k * stride;
      if (i < n_amps) {
        const C2 a = p[i], b = q[i];
        se += a.x * b.x + a.y * b.y;
        sn += a.x * a.x + a.y * a.y;
      }
    }
    ae.add(se);
    an.add(sn);
  }
  const double e = block_sum(ae.value(), red);
  const double nn = block_sum(an.value(), red);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = e;
    partial[2 * blockIdx.x + 1] = nn;
  }
}

// ------------------------------------------------------------------ reverse sweep

template <typename R, bool STREAM, int TT, bool GUARD>
__global__ void __launch_bounds__(NT, 2) k_reverse(R *psi, R *lam, int n, PassDesc pd,
                                                   const GroupDesc *groups,
                                                   const typename Vec2<R>::type *lut,
                                                   const uint64_t *signmask, const R *wlut,
                                                   double *partial) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  constexpr int P = PairShape<TT, GUARD>::P;
  extern __shared__ __align__(16) unsigned char smem[];
  PassDesc pq = pd;
  pq.b_begin = pq.b_end = 0;
  const SmemLayout L =
      smem_layout(sizeof(C2), pq, 2, sizeof(double) * RP_MAX + sizeof(R) * (NT / 32) * M_MAX);
  const Stage<R> st = stage_pass<R>(smem, pq, L, groups, nullptr, lut);
  C2 *tp = reinterpret_cast<C2 *>(smem + L.tiles);
  C2 *tl = tp + st.amps;
  double *acc = reinterpret_cast<double *>(smem + L.extra);   // [RP_MAX]
  R *wpart = reinterpret_cast<R *>(acc + RP_MAX);             // [NT/32][M_MAX]
  const int nrot = pd.rot_end - pd.rot_begin;
  for (int k = threadIdx.x; k < nrot; k += NT) acc[k] = 0.0;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const int ng = pd.g_end - pd.g_begin;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(t, pd.umask);
    load_tile<R, STREAM>(psi, base, st, reinterpret_cast<V *>(tp));
    load_tile<R, STREAM>(lam, base, st, reinterpret_cast<V *>(tl));
    tile_codes(st, ng, t);
    __syncthreads();
    for (int k = ng - 1; k >= 0; --k) {
      const GroupDesc &d = st.gs[k];
      const C2 *lt = st.lut + d.lut;
      const int kind = d.kind;
      // One-parameter groups accumulate sum_pairs w(code) val, w = sum_k coef_k sign_k(code),
      // in one slot (credited to the group's first rotation); others one slot per rotation.
      const bool one = d.one_param != 0;
      const int m = one ? 1 : d.m;
      const R *wl = wlut + d.wlut;
      const int rot0 = (int)d.rot0;
      const uint64_t *sm = signmask + pd.rot_begin + rot0;
      const uint32_t code0 = st.tcode[k] ^ d.plane[lane] ^ d.pwarp[warp];
      uint64_t mask[M_MAX];
      R a_k[M_MAX];
#pragma unroll
      for (int q = 0; q < M_MAX; ++q) {
        mask[q] = (!one && q < m) ? __ldg(&sm[q]) : 0ull;
        a_k[q] = 0;
      }
      if (kind == KIND_DIAG) {
#pragma unroll
        for (int j = 0; j < 2 * P; ++j) {
          const uint32_t l = tid + NT * j;
          if (GUARD && l >= st.amps) break;
          const uint32_t code = code0 ^ d.pjcode[j];
          const C2 cs = lt[code];
          const C2 a = tp[l], b = tl[l];
          const R val = b.x * a.y - b.y * a.x;   // Im(conj(lam) psi)
          if (one) {
            a_k[0] += __ldg(wl + code) * val;
          } else {
#pragma unroll
            for (int q = 0; q < M_MAX; ++q)
              if (q < m) a_k[q] += ((mask[q] >> code) & 1) ? -val : val;
          }
          C2 a2 = a, b2 = b;
          phase(a2, cs.x, -cs.y);
          phase(b2, cs.x, -cs.y);
          tp[l] = a2;
          tl[l] = b2;
        }
      } else if (!GUARD || tid < (st.amps >> 1)) {
        const uint32_t li0 = insert_zero(tid, d.pivot);
        const uint32_t xl = d.xl;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const uint32_t li = li0 | d.pu[j], lj = li ^ xl;
          const uint32_t code = code0 ^ d.pjcode[j];
          const C2 cs = lt[code];
          C2 pa = tp[li], pb = tp[lj], la = tl[li], lb = tl[lj];
          R val;
          if (kind == KIND_REAL) {
            // Re(conj(lam_j) psi_i - conj(lam_i) psi_j)
            val = (lb.x * pa.x + lb.y * pa.y) - (la.x * pb.x + la.y * pb.y);
          } else {
            // Im(conj(lam_i) psi_j + conj(lam_j) psi_i)
            val = (la.x * pb.y - la.y * pb.x) + (lb.x * pa.y - lb.y * pa.x);
          }
          if (one) {
            a_k[0] += __ldg(wl + code) * val;
          } else {
#pragma unroll
            for (int q = 0; q < M_MAX; ++q)
              if (q < m) a_k[q] += ((mask[q] >> code) & 1) ? -val : val;
          }
          if (kind == KIND_REAL) {
            rot_real(pa, pb, cs.x, -cs.y);
            rot_real(la, lb, cs.x, -cs.y);
          } else {
            rot_xrot(pa, pb, cs.x, -cs.y);
            rot_xrot(la, lb, cs.x, -cs.y);
          }
          tp[li] = pa;
          tp[lj] = pb;
          tl[li] = la;
          tl[lj] = lb;
        }
      }
      // warp sums -> smem -> fixed-order CTA sum into acc (double)
#pragma unroll
      for (int q = 0; q < M_MAX; ++q) {
        if (q < m) {
          R v = a_k[q];
          for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
          if (lane == 0) wpart[warp * M_MAX + q] = v;
        }
      }
      __syncthreads();
      if ((int)threadIdx.x < m) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += (double)wpart[w * M_MAX + threadIdx.x];
        acc[rot0 + threadIdx.x] += s;
      }
      __syncthreads();
    }
    store_tile<R, STREAM>(psi, base, st, reinterpret_cast<const V *>(tp));
    store_tile<R, STREAM>(lam, base, st, reinterpret_cast<const V *>(tl));
    __syncthreads();
  }
  for (int k = threadIdx.x; k < nrot; k += NT) partial[(size_t)blockIdx.x * RP_MAX + k] = acc[k];
}

// ------------------------------------------------------------------ register-blocked reverse sweep
//
// Passes whose groups each share one parameter (every UCCSD excitation) run
// Algorithm 1's reverse loop on the sweep's register blocks: a thread holds
// one coset of psi and of lambda, walks the block's groups backwards, and for
// each group adds w(code) * val over its pairs (val the pair's part of
// Im<lambda|P|psi>, w = sum_k coef_k sign_k(code) the group's gradient
// weight), then undoes the group on both vectors.  A group's sum is
// warp-reduced and kept per warp in shared memory across tiles; at the end of
// the pass the warps are added in fixed order and the sum is credited to the
// group's first rotation.  complex64 only (two 16-amplitude cosets fit in
// registers); other passes use k_reverse.  The weights are staged beside the
// LUT with the same entry indices, so both are addressed by XOR.

// inverse of rot_real: [[c, s], [-s, c]] with e = (c, c, s, s)
__device__ __forceinline__ void rot_real_inv(float2 &a, float2 &b, float4 e) {
  const unsigned long long A = f2_pack(a.x, a.y), B = f2_pack(b.x, b.y);
  const unsigned long long C = f2_pack(e.x, e.y), S = f2_pack(e.z, e.w);
  const unsigned long long na = f2_fma(S, B, f2_mul(C, A));
  const unsigned long long nb = f2_sub(f2_mul(C, B), f2_mul(S, A));
  a = f2_unpack(na);
  b = f2_unpack(nb);
}

// Pairs (c, c ^ A) of one group: weighted gradient sum, then the group undone on psi (v) and lambda (u).
template <int D, int A, int KIND>
__device__ __forceinline__ float rev_pairs(float2 (&v)[1 << D], float2 (&u)[1 << D], const unsigned char *base,
                                           uint32_t lp, uint32_t wp, const uint32_t (&G)[D],
                                           const uint32_t (&Gw)[D]) {
  constexpr int HB = 31 - __builtin_clz(A);
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    if ((c >> HB) & 1) continue;
    const float4 e = *reinterpret_cast<const float4 *>(base + combo_off<D>(lp, G, c));
    const float w = *reinterpret_cast<const float *>(base + combo_off<D>(wp, Gw, c));
    const float2 pa = v[c], pb = v[c ^ A], la = u[c], lb = u[c ^ A];
    float val;
    if (KIND == KIND_REAL) val = (lb.x * pa.x + lb.y * pa.y) - (la.x * pb.x + la.y * pb.y);
    else val = (la.x * pb.y - la.y * pb.x) + (lb.x * pa.y - lb.y * pa.x);
    acc += w * val;
    if (KIND == KIND_REAL) {
      rot_real_inv(v[c], v[c ^ A], e);
      rot_real_inv(u[c], u[c ^ A], e);
    } else {
      rot_xrot(v[c], v[c ^ A], e.x, -e.z);
      rot_xrot(u[c], u[c ^ A], e.x, -e.z);
    }
  }
  return acc;
}

template <int D, int KIND>
__device__ __forceinline__ float rev_pairs_sw(int a, float2 (&v)[1 << D], float2 (&u)[1 << D],
                                              const unsigned char *base, uint32_t lp, uint32_t wp,
                                              const uint32_t (&G)[D], const uint32_t (&Gw)[D]) {
  switch (a) {
#define Q2_RC(X) \
  case X:        \
    if constexpr (X < (1 << D)) return rev_pairs<D, X, KIND>(v, u, base, lp, wp, G, Gw); \
    break;
    Q2_RC(1) Q2_RC(2) Q2_RC(3) Q2_RC(4) Q2_RC(5) Q2_RC(6) Q2_RC(7) Q2_RC(8)
    Q2_RC(9) Q2_RC(10) Q2_RC(11) Q2_RC(12) Q2_RC(13) Q2_RC(14) Q2_RC(15)
#undef Q2_RC
    default: break;
  }
  return 0.f;
}

struct RevStage {
  uint32_t w_off;   // byte offset (from the start of shared memory) of the staged weights
  double *wacc;     // [NT/32][G_STAGE] per-warp group sums
};

// Group k of a canonical block (pairs along basis bit k, REAL): gradient sum and undo.
template <int D, int K>
__device__ __forceinline__ float rev_canon_group(float2 (&v)[1 << D], float2 (&u)[1 << D],
                                                 const Stage<float, float4> &s, const RevStage &rs, int gi,
                                                 uint32_t cb, int lut_begin) {
  constexpr int ES = log2_int(sizeof(float4));
  const GroupDesc &g = s.gs[gi];
  const uint32_t rel = g.lut - (uint32_t)lut_begin;
  const uint32_t goff = (uint32_t)(reinterpret_cast<const unsigned char *>(s.lut + g.lut) - s.base);
  uint32_t G[D], Gw[D];
  group_gens<D, ES>(g, K, G);
#pragma unroll
  for (int i = 0; i < D; ++i) Gw[i] = G[i] >> (ES - 2);
  return rev_pairs<D, 1 << K, KIND_REAL>(v, u, s.base, goff | (cb << ES), (rs.w_off + (rel << 2)) | (cb << 2), G,
                                         Gw);
}

// Canonical groups K, K-1, ..., 0 of a block, in that order (the reverse of the sweep's order).
template <int D, int K>
__device__ __forceinline__ void rev_canon(float2 (&v)[1 << D], float2 (&u)[1 << D], const Stage<float, float4> &s,
                                          const RevStage &rs, int gb, uint32_t lane, uint32_t warp, int j,
                                          int lut_begin) {
  if constexpr (K >= 0) {
    const int gi = gb + K;
    const GroupDesc &g = s.gs[gi];
    const uint32_t cb = s.tcode[gi] ^ g.blane[lane] ^ g.bwarp[warp] ^ g.bjcode[j];
    float acc = rev_canon_group<D, K>(v, u, s, rs, gi, cb, lut_begin);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) rs.wacc[warp * G_STAGE + gi] += (double)acc;
    rev_canon<D, K - 1>(v, u, s, rs, gb, lane, warp, j, lut_begin);
  }
}

template <int D, int J>
__device__ __forceinline__ void reverse_block(float2 *tp, float2 *tl, const BlockDesc &B,
                                              const Stage<float, float4> &s, const RevStage &rs, int lut_begin) {
  constexpr int N = 1 << D;
  constexpr int ES = log2_int(sizeof(float4));
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t bt = tid;
#pragma unroll
  for (int i = 0; i < D; ++i) bt = insert_zero(bt, B.piv[i]);
  const int gb = B.g_begin, ge = B.g_end;
  unsigned char *pbase = reinterpret_cast<unsigned char *>(tp);
  unsigned char *lbase = reinterpret_cast<unsigned char *>(tl);
  uint32_t W[D];
#pragma unroll
  for (int i = 0; i < D; ++i) W[i] = (uint32_t)B.comb[1 << i] << 3;
#pragma unroll 1
  for (int j = 0; j < J; ++j) {
    const uint32_t o0 = (bt ^ B.uj[j]) << 3;
    float2 v[N], u[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
      v[c] = *reinterpret_cast<const float2 *>(pbase + combo_off<D>(o0, W, c));
      u[c] = *reinterpret_cast<const float2 *>(lbase + combo_off<D>(o0, W, c));
    }
    const bool canon = B.canon == D;
    const int g_stop = canon ? gb + D : gb;   // canonical leading groups go last, unrolled
#pragma unroll 1
    for (int gi = ge - 1; gi >= g_stop; --gi) {
      const GroupDesc &g = s.gs[gi];
      const uint32_t cb = s.tcode[gi] ^ g.blane[lane] ^ g.bwarp[warp] ^ g.bjcode[j];
      const uint32_t rel = g.lut - (uint32_t)lut_begin;   // entry index in the staged LUT and weights
      const uint32_t goff = (uint32_t)(reinterpret_cast<const unsigned char *>(s.lut + g.lut) - s.base);
      const uint32_t lp = goff | (cb << ES);
      const uint32_t wp = (rs.w_off + (rel << 2)) | (cb << 2);
      uint32_t G[D], Gw[D];
      group_gens<D, ES>(g, -1, G);
#pragma unroll
      for (int i = 0; i < D; ++i) Gw[i] = G[i] >> (ES - 2);
      float acc;
      if (g.kind == KIND_REAL) {
        acc = rev_pairs_sw<D, KIND_REAL>(g.a, v, u, s.base, lp, wp, G, Gw);
      } else if (g.kind == KIND_XROT) {
        acc = rev_pairs_sw<D, KIND_XROT>(g.a, v, u, s.base, lp, wp, G, Gw);
      } else {
        acc = 0.f;
#pragma unroll
        for (int c = 0; c < N; ++c) {
          const float4 e = *reinterpret_cast<const float4 *>(s.base + combo_off<D>(lp, G, c));
          const float w = *reinterpret_cast<const float *>(s.base + combo_off<D>(wp, Gw, c));
          acc += w * (u[c].x * v[c].y - u[c].y * v[c].x);
          phase(v[c], e.x, -e.z);
          phase(u[c], e.x, -e.z);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) rs.wacc[warp * G_STAGE + gi] += (double)acc;
    }
    if (canon) rev_canon<D, D - 1>(v, u, s, rs, gb, lane, warp, j, lut_begin);
    uint32_t W2[D];   // reloaded rather than kept live across the group loop
#pragma unroll
    for (int i = 0; i < D; ++i) W2[i] = (uint32_t)B.comb[1 << i] << 3;
#pragma unroll
    for (int c = 0; c < N; ++c) {
      *reinterpret_cast<float2 *>(pbase + combo_off<D>(o0, W2, c)) = v[c];
      *reinterpret_cast<float2 *>(lbase + combo_off<D>(o0, W2, c)) = u[c];
    }
  }
}

template <int TT>
__device__ __forceinline__ void reverse_block_any(float2 *tp, float2 *tl, const BlockDesc &B,
                                                  const Stage<float, float4> &s, const RevStage &rs,
                                                  int lut_begin) {
  switch (B.d) {
    case 1: reverse_block<1, BlockShape<TT, 1>::J>(tp, tl, B, s, rs, lut_begin); break;
    case 2:
      if constexpr (TT >= 10) reverse_block<2, BlockShape<TT, 2>::J>(tp, tl, B, s, rs, lut_begin);
      break;
    case 3:
      if constexpr (TT >= 11) reverse_block<3, BlockShape<TT, 3>::J>(tp, tl, B, s, rs, lut_begin);
      break;
    case 4:
      if constexpr (TT >= 12) reverse_block<4, BlockShape<TT, 4>::J>(tp, tl, B, s, rs, lut_begin);
      break;
  }
}

// Extra shared memory of k_reverse_blk after the staged tables: weights (one
// float per LUT entry, 256-byte aligned) and the per-warp group sums.
__host__ __device__ inline size_t rev_extra_bytes(int lut_count) {
  return 256 + align16(sizeof(float) * (size_t)lut_count) + sizeof(double) * (NT / 32) * G_STAGE;
}

template <int TT>
__global__ void __launch_bounds__(NT, 2) k_reverse_blk(float *psi, float *lam, int n, PassDesc pd,
                                                       const GroupDesc *groups, const BlockDesc *blocks,
                                                       const float2 *lut, const float *wlut, double *partial) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(sizeof(float2), pd, 2, rev_extra_bytes(pd.lut_count), sizeof(float4),
                                   sizeof(float4) << R_MAX_ROT);
  const Stage<float, float4> st = stage_pass<float, float4>(smem, pd, L, groups, blocks, lut);
  float2 *tp = reinterpret_cast<float2 *>(smem + L.tiles);
  float2 *tl = tp + st.amps;
  const int ng = pd.g_end - pd.g_begin, nb = pd.b_end - pd.b_begin;
  RevStage rs;
  rs.w_off = (uint32_t)((L.extra + 255) & ~(size_t)255);
  float *wst = reinterpret_cast<float *>(smem + rs.w_off);
  rs.wacc = reinterpret_cast<double *>(smem + rs.w_off + align16(sizeof(float) * (size_t)pd.lut_count));
  for (int i = threadIdx.x; i < (NT / 32) * G_STAGE; i += NT) rs.wacc[i] = 0.0;
  __syncthreads();   // group descriptors are staged by other warps' 16-byte copies
  for (int g = threadIdx.x; g < ng; g += NT) {   // weights beside the LUT entries of each group
    const GroupDesc &d = st.gs[g];
    const uint32_t rel = d.lut - (uint32_t)pd.lut_begin;
    for (int c = 0; c < (1 << d.r); ++c) wst[rel + c] = __ldg(wlut + d.wlut + c);
  }
  __syncthreads();
  using V = typename Vec16<float>::type;
  const uint64_t ntiles = 1ull << (n - pd.T);
  TileWalk tw(blockIdx.x, gridDim.x, pd.umask);
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, tw.next()) {
    const uint64_t base = tw.base;
    async_load_tile(psi, base, st, tp);
    async_load_tile(lam, base, st, tl);
    tile_codes(st, ng, t);
    cp_async_wait_all();
    __syncthreads();
    for (int b = nb - 1; b >= 0; --b) {
      reverse_block_any<TT>(tp, tl, st.bs[b], st, rs, pd.lut_begin);
      __syncthreads();
    }
    store_tile<float, false>(psi, base, st, reinterpret_cast<const V *>(tp));
    store_tile<float, false>(lam, base, st, reinterpret_cast<const V *>(tl));
    __syncthreads();   // every thread has read its pieces before the next tiles land
  }
  // per-rotation partials of this CTA: group sums at each group's first rotation, zero elsewhere
  const int nrot = pd.rot_end - pd.rot_begin;
  for (int k = threadIdx.x; k < nrot; k += NT) partial[(size_t)blockIdx.x * RP_MAX + k] = 0.0;
  __syncthreads();
  for (int g = threadIdx.x; g < ng; g += NT) {
    double sum = 0.0;
    for (int w = 0; w < NT / 32; ++w) sum += rs.wacc[w * G_STAGE + g];
    partial[(size_t)blockIdx.x * RP_MAX + st.gs[g].rot0] = sum;
  }
}

// g[k] = sum_b partial[b][k], fixed order over b.
__global__ void k_reduce_rot(const double *partial, int nblocks, int nrot, double *g) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nrot) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * RP_MAX + k];
  g[k] = s;
}

// ------------------------------------------------------------------ launchers

namespace {

int sm_count() {
  static int cached = -1, cached_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (cached < 0 || cached_dev != dev) {
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    cached_dev = dev;
  }
  return cached;
}

template <typename K>
int blocks_per_sm(K kernel, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, NT, smem) != cudaSuccess) return 1;
  return b > 0 ? b : 1;
}

// Largest dynamic shared memory any pass of a kernel instantiation can ask for
// (tile size T, smallest chunk, fullest staged tables).  The attribute is
// per-function state shared by every host thread, so it is always set to this
// fixed value, never to one launch's size.
size_t worst_smem(int amp_bytes, int T, int vectors, size_t extra, int lut_entry_bytes = 0,
                  size_t lut_align = 16, int lut_max = LUT_STAGE) {
  if (lut_entry_bytes == 0) lut_entry_bytes = amp_bytes;
  PassDesc pd{};
  pd.T = T <= 8 ? 8 : T;
  pd.C = 1;
  pd.g_begin = 0;
  pd.g_end = G_STAGE;
  pd.b_begin = 0;
  pd.b_end = G_STAGE;
  pd.lut_count = lut_max;
  SmemLayout L;
  size_t o = 0;
  o = align16(o + (size_t)amp_bytes * ((size_t)1 << pd.T) * vectors);
  o = align16(o + sizeof(uint64_t) * ((size_t)1 << (pd.T - pd.C)));
  o = align16(o + sizeof(GroupDesc) * G_STAGE);
  o = align16(o + sizeof(BlockDesc) * G_STAGE);
  o = align_to(o, lut_align);
  o = align16(o + (size_t)lut_entry_bytes * lut_max);
  o = align16(o + sizeof(uint32_t) * G_STAGE);
  o = align16(o + extra);
  (void)L;
  return o;
}

// The shared-memory attribute is per-function state shared by every host
// thread: it is set once per device and function, under a lock, so no
// launch on another thread ever overlaps a change of it.
template <typename K>
cudaError_t prepare(K kernel, size_t smem_cap) {
  if (smem_cap <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::set<std::pair<int, const void *>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const std::pair<int, const void *> key(dev, reinterpret_cast<const void *>(kernel));
  std::lock_guard<std::mutex> g(mu);
  if (done.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap);
  if (e == cudaSuccess) done.insert(key);
  return e;
}

unsigned grid_for(uint64_t ntiles, int per_sm) {
  const uint64_t cap = (uint64_t)sm_count() * (uint64_t)per_sm;
  return (unsigned)(ntiles < cap ? ntiles : cap);
}

bool streaming(int n, int bytes) { return ((uint64_t)bytes << n) > (64ull << 20); }

// Pick the kernel instantiation for a pass's tile size T (9..13; smaller tiles are guarded).
#define Q2_DISPATCH(KERNEL, R, n, T)                                                      \
  [&]() -> decltype(&KERNEL<R, true, 9, true>) {                                        \
    const bool st_ = streaming(n, 2 * (int)sizeof(R));                                  \
    switch (T) {                                                                          \
      case 9: return st_ ? &KERNEL<R, true, 9, false> : &KERNEL<R, false, 9, false>;     \
      case 10: return st_ ? &KERNEL<R, true, 10, false> : &KERNEL<R, false, 10, false>;  \
      case 11: return st_ ? &KERNEL<R, true, 11, false> : &KERNEL<R, false, 11, false>;  \
      case 12: return st_ ? &KERNEL<R, true, 12, false> : &KERNEL<R, false, 12, false>;  \
      case 13: return st_ ? &KERNEL<R, true, 13, false> : &KERNEL<R, false, 13, false>;  \
      default: return st_ ? &KERNEL<R, true, 9, true> : &KERNEL<R, false, 9, true>;      \
    }                                                                                     \
  }()

// Largest LUT of a Hamiltonian pass for a dtype (entries staged in shared memory).
template <typename R> constexpr int ham_lut_max() { return sizeof(R) == 4 ? LUT_STAGE_HAM_C64 : LUT_STAGE; }

PassDesc worst_pass(int T, int C) {
  PassDesc pd{};
  pd.T = T;
  pd.C = C;
  pd.g_begin = 0;
  pd.g_end = G_STAGE;
  pd.b_begin = 0;
  pd.b_end = G_STAGE;
  pd.lut_count = LUT_STAGE;
  return pd;
}

}  // namespace

// Probe of the bounded wait: an mbarrier that nothing completes (one pending
// arrival, no copies), waited on with `polls` polls; the wait gives up and
// records itself exactly like a tile-copy wait that never completes.
__global__ void k_wait_probe(uint32_t polls, unsigned *fault) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0, fault, polls);
}

cudaError_t launch_wait_probe(uint32_t polls, unsigned *fault, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(polls, fault);
  return cudaGetLastError();
}

// Give-ups of the asynchronous calls on the current device: read, then cleared
// (stream-ordered on st; the caller synchronizes st before using *host).
cudaError_t take_async_faults(unsigned *host, cudaStream_t st) {
  static const unsigned zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(host, g_async_faults, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(g_async_faults, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, st);
  return e;
}

// FP64 FMA throughput probe: each thread runs 8 independent chains of `iters`
// fused multiply-adds (2 flops each) on values that stay finite (|a| < 1).
__global__ void __launch_bounds__(NT) k_fp64_rate(int iters, double seed, double *sink) {
  double v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = seed * (double)(threadIdx.x + k + 1) * 1e-6;
  const double a = 0.999999, b = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
  }
  double t = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += v[k];
  if (t == 12345.0) sink[0] = t;   // keeps the chains live; never true for these values
}

cudaError_t measure_fp64_rate(double *flops_per_s, cudaStream_t st) {
  const int blocks = sm_count() * 2, iters = 1 << 11;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  k_fp64_rate<<<blocks, NT, 0, st>>>(16, 0.5, nullptr);   // warm-up
  cudaEventRecord(e0, st);
  k_fp64_rate<<<blocks, NT, 0, st>>>(iters, 0.5, nullptr);
  cudaEventRecord(e1, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) *flops_per_s = (double)blocks * NT * iters * 8 * 2 / (ms * 1e-3);
  return e;
}

size_t tile_smem_bytes(int amp_bytes, int T, int C, int vectors) {
  PassDesc wp = worst_pass(T, C);
  wp.lut_count = amp_bytes == 8 ? LUT_STAGE_HAM_C64 : LUT_STAGE;
  return smem_layout(amp_bytes, wp, vectors, sizeof(double) * (NT / 32), amp_bytes, (size_t)amp_bytes << R_MAX).total;
}

size_t reverse_smem_bytes(int amp_bytes, int T, int C) {
  PassDesc pd = worst_pass(T, C);
  pd.b_end = 0;
  return smem_layout(amp_bytes, pd, 2, sizeof(double) * RP_MAX + (size_t)(amp_bytes / 2) * (NT / 32) * M_MAX)
      .total;
}

int max_grid_blocks(int amp_bytes, int T) {
  (void)amp_bytes;
  (void)T;
  return sm_count() * 8;
}

template <typename R>
cudaError_t launch_init_hf(R *psi, int n, int n_elec, cudaStream_t st) {
  const uint64_t n_amps = 1ull << n;
  const uint64_t nv = (n_amps + Vec16<R>::amps - 1) / Vec16<R>::amps;
  uint64_t blocks = (nv + NT - 1) / NT;
  const uint64_t cap = (uint64_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  k_init_hf<R><<<(unsigned)blocks, NT, 0, st>>>(psi, n_amps, (1ull << n_elec) - 1);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sweep(R *psi, int n, const PassDesc &pd, const GroupDesc *groups,
                         const BlockDesc *blocks, const void *lut, unsigned *fault, bool c4, cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  const int nvec = 1;
  const int eb = (int)sizeof(typename SweepLut<R>::E);
  if constexpr (sizeof(R) == 4 && Q2_F32X2) {
    if (c4 && (pd.T == 12 || pd.T == 13) && pd.g_end - pd.g_begin <= C4_MAX_GROUPS) {
      const size_t smem =
          smem_layout(sizeof(C2), pd, nvec, c4_extra_bytes(pd.g_end - pd.g_begin, pd.b_end - pd.b_begin), eb,
                      (size_t)eb << R_MAX_ROT, (size_t)eb << R_MAX_ROT).total;
      const bool st_ = streaming(n, 2 * (int)sizeof(R));
      auto k = pd.T == 12 ? (st_ ? &k_sweep_c4<true, 12> : &k_sweep_c4<false, 12>)
                          : (st_ ? &k_sweep_c4<true, 13> : &k_sweep_c4<false, 13>);
      PassDesc wp = worst_pass(pd.T, pd.C);
      wp.g_end = C4_MAX_GROUPS;
      wp.b_end = C4_MAX_GROUPS / 4;
      cudaError_t e = prepare(k, smem_layout(sizeof(C2), wp, nvec, c4_extra_bytes(C4_MAX_GROUPS, C4_MAX_GROUPS / 4),
                                             eb, (size_t)eb << R_MAX_ROT, (size_t)eb << R_MAX_ROT).total);
      if (e != cudaSuccess) return e;
      const unsigned grid = grid_for(1ull << (n - pd.T), blocks_per_sm(k, smem));
      k<<<grid, NT, smem, st>>>(reinterpret_cast<float *>(psi), n, pd, groups, blocks,
                                reinterpret_cast<const float2 *>(lut));
      return cudaGetLastError();
    }
  }
  const size_t smem = smem_layout(sizeof(C2), pd, nvec, 0, eb, (size_t)eb << R_MAX_ROT).total;
  auto k = Q2_DISPATCH(k_sweep, R, n, pd.T);
  cudaError_t e = prepare(k, worst_smem(sizeof(C2), pd.T, nvec, 0, eb, (size_t)eb << R_MAX_ROT));
  if (e != cudaSuccess) return e;
  const unsigned grid = grid_for(1ull << (n - pd.T), blocks_per_sm(k, smem));
  k<<<grid, NT, smem, st>>>(psi, n, pd, groups, blocks, reinterpret_cast<const C2 *>(lut), fault);
  return cudaGetLastError();
}

template <typename R>
int expect_grid(int n, int T, int C) {
  using C2 = typename Vec2<R>::type;
  const int nvec = 1;
  const size_t smem = tile_smem_bytes(sizeof(C2), T, C, nvec);
  auto k = Q2_DISPATCH(k_expect, R, n, T);
  prepare(k, worst_smem(sizeof(C2), T, nvec, sizeof(double) * (NT / 32), sizeof(C2), sizeof(C2) << R_MAX,
                        ham_lut_max<R>()));
  return (int)grid_for(1ull << (n - T), blocks_per_sm(k, smem));
}

template <typename R>
cudaError_t launch_expect(const R *psi, int n, const PassDesc &pd, const GroupDesc *groups,
                          const BlockDesc *blocks, const void *lut, double *partial, int grid, bool first,
                          unsigned *fault, bool lean, cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  const int nvec = 1;
  if constexpr (sizeof(R) == 4) {
    if (lean && (pd.T == 12 || pd.T == 13)) {
      const int ng = pd.g_end - pd.g_begin;
      const size_t smem = smem_layout(sizeof(C2), pd, nvec, efast_extra_bytes(ng), sizeof(C2), sizeof(C2) << R_MAX,
                                      sizeof(C2) << R_MAX).total;
      const bool st_ = streaming(n, 2 * (int)sizeof(R));
      auto k = pd.T == 12 ? (st_ ? &k_expect_fast<true, 12> : &k_expect_fast<false, 12>)
                          : (st_ ? &k_expect_fast<true, 13> : &k_expect_fast<false, 13>);
      cudaError_t e = prepare(k, worst_smem(sizeof(C2), pd.T, nvec, efast_extra_bytes(G_STAGE) + (sizeof(C2) << R_MAX),
                                            sizeof(C2), sizeof(C2) << R_MAX, ham_lut_max<R>()));
      if (e != cudaSuccess) return e;
      k<<<grid, NT, smem, st>>>(reinterpret_cast<const float *>(psi), n, pd, groups, blocks,
                                reinterpret_cast<const float2 *>(lut), partial, first ? 1 : 0);
      return cudaGetLastError();
    }
  }
  const size_t smem =
      smem_layout(sizeof(C2), pd, nvec, sizeof(double) * (NT / 32), sizeof(C2), sizeof(C2) << R_MAX).total;
  auto k = Q2_DISPATCH(k_expect, R, n, pd.T);
  cudaError_t e = prepare(k, worst_smem(sizeof(C2), pd.T, nvec, sizeof(double) * (NT / 32), sizeof(C2),
                                        sizeof(C2) << R_MAX, ham_lut_max<R>()));
  if (e != cudaSuccess) return e;
  k<<<grid, NT, smem, st>>>(psi, n, pd, groups, blocks, reinterpret_cast<const C2 *>(lut), partial,
                            first ? 1 : 0, fault);
  return cudaGetLastError();
}

cudaError_t launch_reduce_pairs(const double *partial, int nblocks, double *out, cudaStream_t st) {
  k_reduce_pairs<<<1, NT, 0, st>>>(partial, nblocks, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_happly(const R *psi, R *lam, int n, const PassDesc &pd, const GroupDesc *groups,
                          const BlockDesc *blocks, const void *lut, bool first, unsigned *fault,
                          cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  if (blocks && pd.T >= 9 && pd.T <= T_LIMIT) {   // register-blocked path
    const size_t al = sizeof(C2) << R_MAX;
    const size_t smem = smem_layout(sizeof(C2), pd, 2, 0, sizeof(C2), al).total;
    decltype(&k_happly_blk<R, 9>) k;
    switch (pd.T) {
      case 9: k = &k_happly_blk<R, 9>; break;
      case 10: k = &k_happly_blk<R, 10>; break;
      case 11: k = &k_happly_blk<R, 11>; break;
      case 12: k = &k_happly_blk<R, 12>; break;
      default: k = &k_happly_blk<R, 13>; break;
    }
    cudaError_t e = prepare(k, worst_smem(sizeof(C2), pd.T, 2, 0, sizeof(C2), al, ham_lut_max<R>()));
    if (e != cudaSuccess) return e;
    const unsigned grid = grid_for(1ull << (n - pd.T), blocks_per_sm(k, smem));
    k<<<grid, NT, smem, st>>>(psi, lam, n, pd, groups, blocks, reinterpret_cast<const C2 *>(lut), first ? 1 : 0);
    return cudaGetLastError();
  }
  PassDesc pq = pd;
  pq.b_begin = pq.b_end = 0;
  const size_t smem = smem_layout(sizeof(C2), pq, 2, 0).total;
  auto k = Q2_DISPATCH(k_happly, R, n, pd.T);
  cudaError_t e = prepare(k, worst_smem(sizeof(C2), pd.T, 2, 0, 0, 16, ham_lut_max<R>()));
  if (e != cudaSuccess) return e;
  const unsigned grid = grid_for(1ull << (n - pd.T), blocks_per_sm(k, smem));
  k<<<grid, NT, smem, st>>>(psi, lam, n, pd, groups, reinterpret_cast<const C2 *>(lut), first ? 1 : 0);
  return cudaGetLastError();
}

template <typename R>
int dot_grid(int n) {
  const uint64_t n_amps = 1ull << n;
  uint64_t blocks = (n_amps + NT - 1) / NT;
  const uint64_t cap = (uint64_t)sm_count() * 4;
  return (int)(blocks < cap ? blocks : cap);
}

template <typename R>
cudaError_t launch_dot(const R *psi, const R *lam, int n, double *partial, int grid, cudaStream_t st) {
  k_dot<R><<<grid, NT, 0, st>>>(psi, lam, 1ull << n, partial);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_reverse(R *psi, R *lam, int n, const PassDesc &pd, const GroupDesc *groups,
                           const BlockDesc *blocks, bool one_param, const void *lut, const uint64_t *signmask,
                           const R *wlut, double *partial, double *gphi, unsigned *fault, cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  if constexpr (sizeof(R) == 4) {
    if (one_param && pd.T >= 9 && pd.T <= T_LIMIT) {   // register-blocked path (complex64)
      const size_t eb = sizeof(float4), al = eb << R_MAX_ROT;
      const size_t smem = smem_layout(sizeof(float2), pd, 2, rev_extra_bytes(pd.lut_count), (int)eb, al).total;
      decltype(&k_reverse_blk<9>) k;
      switch (pd.T) {
        case 9: k = &k_reverse_blk<9>; break;
        case 10: k = &k_reverse_blk<10>; break;
        case 11: k = &k_reverse_blk<11>; break;
        case 12: k = &k_reverse_blk<12>; break;
        default: k = &k_reverse_blk<13>; break;
      }
      cudaError_t e = prepare(k, worst_smem(sizeof(float2), pd.T, 2, rev_extra_bytes(LUT_STAGE), (int)eb, al));
      if (e != cudaSuccess) return e;
      const unsigned grid = grid_for(1ull << (n - pd.T), blocks_per_sm(k, smem));
      k<<<grid, NT, smem, st>>>(psi, lam, n, pd, groups, blocks, reinterpret_cast<const float2 *>(lut), wlut,
                                partial);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      const int nrot = pd.rot_end - pd.rot_begin;
      k_reduce_rot<<<(nrot + 127) / 128, 128, 0, st>>>(partial, (int)grid, nrot, gphi + pd.rot_begin);
      return cudaGetLastError();
    }
  }
  PassDesc pq = pd;
  pq.b_begin = pq.b_end = 0;
  const size_t smem =
      smem_layout(sizeof(C2), pq, 2, sizeof(double) * RP_MAX + sizeof(R) * (NT / 32) * M_MAX).total;
  auto k = Q2_DISPATCH(k_reverse, R, n, pd.T);
  cudaError_t e = prepare(k, worst_smem(sizeof(C2), pd.T, 2, sizeof(double) * RP_MAX + sizeof(R) * (NT / 32) * M_MAX));
  if (e != cudaSuccess) return e;
  const unsigned grid = grid_for(1ull << (n - pd.T), blocks_per_sm(k, smem));
  k<<<grid, NT, smem, st>>>(psi, lam, n, pd, groups, reinterpret_cast<const C2 *>(lut), signmask, wlut, partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nrot = pd.rot_end - pd.rot_begin;
  k_reduce_rot<<<(nrot + 127) / 128, 128, 0, st>>>(partial, (int)grid, nrot, gphi + pd.rot_begin);
  return cudaGetLastError();
}

#define Q2_INST(R)                                                                                  \
  template cudaError_t launch_init_hf<R>(R *, int, int, cudaStream_t);                             \
  template cudaError_t launch_sweep<R>(R *, int, const PassDesc &, const GroupDesc *,              \
                                       const BlockDesc *, const void *, unsigned *, bool,           \
                                       cudaStream_t);                                               \
  template int expect_grid<R>(int, int, int);                                                       \
  template cudaError_t launch_expect<R>(const R *, int, const PassDesc &, const GroupDesc *,        \
                                        const BlockDesc *, const void *, double *, int, bool,       \
                                        unsigned *, bool, cudaStream_t);                            \
  template cudaError_t launch_happly<R>(const R *, R *, int, const PassDesc &, const GroupDesc *,   \
                                        const BlockDesc *, const void *, bool, unsigned *,          \
                                        cudaStream_t);                                              \
  template int dot_grid<R>(int);                                                                    \
  template cudaError_t launch_dot<R>(const R *, const R *, int, double *, int, cudaStream_t);       \
  template cudaError_t launch_reverse<R>(R *, R *, int, const PassDesc &, const GroupDesc *,        \
                                         const BlockDesc *, bool, const void *, const uint64_t *,   \
                                         const R *, double *, double *, unsigned *, cudaStream_t);

Q2_INST(float)
Q2_INST(double)

}  // namespace q2
