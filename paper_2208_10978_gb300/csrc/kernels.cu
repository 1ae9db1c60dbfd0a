// Tile kernels of the state-vector engine (sm_103a).
//
// Every kernel here is HBM-streaming: a persistent grid walks the 2^(n-T)
// tiles of one pass; each CTA gathers a tile (2^(T-C) chunks of 2^C
// contiguous amplitudes) into shared memory with 16-byte loads, applies all
// groups of the pass there, and writes the tile back (or only reduces it).
// Tiles are cosets of the pass's local subspace W (see q2_internal.h), so a
// pass touches every amplitude exactly once and tiles never overlap.  The
// pass's group descriptors and LUT are staged in shared memory once per CTA.
//
// Work split inside a tile: pair q = tid + NT*j (j < P) of a group with pivot
// p is local index insert_zero(q, p) and its partner ^ xl; P = 2^(T-1)/NT is
// a compile-time constant, so the j loop unrolls and its LUT reads are
// independent.  Tiles smaller than 2 * NT amplitudes take a guarded P = 1.
//
//   k_init_hf     HF determinant (Eq. jw-wfn-map)
//   k_sweep       rotation groups, forward or inverse (product formula after Eq. ucc)
//   k_expect      sum_t c_t <psi|P_t|psi> and <psi|psi> (Eq. qubit-ham-detail)
//   k_happly      lambda = H psi (Algorithm 1, start of the backward pass)
//   k_dot         Re<psi|lambda>, <psi|psi>
//   k_reverse     Algorithm 1's reverse loop over one pass: per-rotation
//                 Im<lambda|P_k|psi>, then psi and lambda un-rotated together
//   k_reduce_*    fixed-order reductions of per-CTA partials (deterministic)
#include <cuda_runtime.h>

#include <cstdint>

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

// [tiles: vectors * 2^T amplitudes][off: 2^(T-C) u64][groups][lut][extra]
struct SmemLayout {
  size_t tiles, off, groups, lut, extra, total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

__host__ __device__ inline SmemLayout smem_layout(int amp_bytes, const PassDesc &pd, int vectors,
                                                  size_t extra_bytes) {
  SmemLayout L;
  size_t o = 0;
  L.tiles = o;
  o = align16(o + (size_t)amp_bytes * ((size_t)1 << pd.T) * vectors);
  L.off = o;
  o = align16(o + sizeof(uint64_t) * ((size_t)1 << (pd.T - pd.C)));
  L.groups = o;
  o = align16(o + sizeof(GroupDesc) * (size_t)(pd.g_end - pd.g_begin));
  L.lut = o;
  o = align16(o + (size_t)amp_bytes * (size_t)pd.lut_count);
  L.extra = o;
  o = align16(o + extra_bytes);
  L.total = o;
  return L;
}

template <typename R> struct Tile {
  using C2 = typename Vec2<R>::type;
  int T, C;
  uint32_t amps;
  uint64_t *off;
  const GroupDesc *gs;   // staged groups of the pass (index g - g_begin)
  const C2 *lut;         // staged LUT (index lut - lut_begin)
};

// Stage offsets, group descriptors and LUT of a pass; caller syncs.
template <typename R>
__device__ __forceinline__ Tile<R> stage_pass(unsigned char *smem, const PassDesc &pd,
                                              const SmemLayout &L, const GroupDesc *groups,
                                              const typename Vec2<R>::type *lut) {
  using C2 = typename Vec2<R>::type;
  Tile<R> t;
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
  const int ng = pd.g_end - pd.g_begin;
  uint4 *gd = reinterpret_cast<uint4 *>(smem + L.groups);
  const uint4 *gsrc = reinterpret_cast<const uint4 *>(groups + pd.g_begin);
  for (int i = threadIdx.x; i < ng * (int)(sizeof(GroupDesc) / 16); i += NT) gd[i] = __ldg(gsrc + i);
  C2 *ld = reinterpret_cast<C2 *>(smem + L.lut);
  for (int i = threadIdx.x; i < pd.lut_count; i += NT) ld[i] = __ldg(lut + pd.lut_begin + i);
  t.gs = reinterpret_cast<const GroupDesc *>(smem + L.groups);
  t.lut = ld - pd.lut_begin;
  return t;
}

__device__ __forceinline__ uint64_t tile_base(uint64_t t, uint64_t umask) { return deposit_bits(t, umask); }

// Gather one tile of `src` into shared memory.
template <typename R, bool STREAM>
__device__ __forceinline__ void load_tile(const R *src, uint64_t base, const Tile<R> &tc,
                                          typename Vec16<R>::type *dst) {
  using V = typename Vec16<R>::type;
  constexpr int A = Vec16<R>::amps;
  const uint32_t nv = tc.amps / A;
  const uint32_t cm = (1u << tc.C) - 1u;
  const V *g = reinterpret_cast<const V *>(src);
  for (uint32_t v0 = 0; v0 < nv; v0 += 8 * NT) {
    V buf[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t v = v0 + k * NT + threadIdx.x;
      if (v < nv) {
        const uint32_t l = v * A;
        const uint64_t i = (base ^ tc.off[l >> tc.C]) | (l & cm);
        buf[k] = ld16<V, STREAM>(g + i / A);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t v = v0 + k * NT + threadIdx.x;
      if (v < nv) dst[v] = buf[k];
    }
  }
}

template <typename R, bool STREAM>
__device__ __forceinline__ void store_tile(R *dstg, uint64_t base, const Tile<R> &tc,
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

// Code of the thread's first element of a group in the current tile.
__device__ __forceinline__ uint32_t thread_code(const GroupDesc &d, int r, uint64_t packed) {
  uint32_t code = 0;
  for (int l = 0; l < r; ++l) code |= (uint32_t)par64(packed & d.bp[l]) << l;
  return code;
}

// Work assignment of one group for a thread: local indices of its P pairs
// (or 2P diagonal amplitudes) and their codes.
template <int P, bool GUARD>
struct PairIter {
  uint32_t li0, code0;
  int pivot;
  __device__ __forceinline__ uint32_t li(int j) const {
    return li0 | insert_zero((uint32_t)(NT * j), pivot);
  }
};

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

// ------------------------------------------------------------------ rotation sweep

// Apply one rotation group (sign +1 forward, -1 inverse) to a shared-memory tile.
template <typename R, int P, bool GUARD>
__device__ __forceinline__ void rot_group(typename Vec2<R>::type *tile, const GroupDesc &d,
                                          const Tile<R> &tc, uint64_t tpacked, R sgn) {
  using C2 = typename Vec2<R>::type;
  const int kind = d.kind;
  const int r = d.r;
  const C2 *lut = tc.lut + d.lut;
  const uint32_t tid = threadIdx.x;
  if (kind == KIND_DIAG) {
    const uint32_t code0 = thread_code(d, r, tpacked | tid);
#pragma unroll
    for (int j = 0; j < 2 * P; ++j) {
      const uint32_t l = tid + NT * j;
      if (GUARD && l >= tc.amps) break;
      const C2 cs = lut[code0 ^ d.jcode[j]];
      const R c = cs.x, s = sgn * cs.y;
      const C2 a = tile[l];
      tile[l] = C2{c * a.x + s * a.y, c * a.y - s * a.x};
    }
    return;
  }
  const int pivot = d.pivot;
  const uint32_t xl = d.xl;
  if (GUARD && tid >= (tc.amps >> 1)) return;
  const uint32_t li0 = insert_zero(tid, pivot);
  const uint32_t code0 = thread_code(d, r, tpacked | li0);
  if (kind == KIND_REAL) {
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const uint32_t li = li0 | insert_zero((uint32_t)(NT * j), pivot), lj = li ^ xl;
      const C2 cs = lut[code0 ^ d.jcode[j]];
      const R c = cs.x, s = sgn * cs.y;
      const C2 a = tile[li], b = tile[lj];
      tile[li] = C2{c * a.x - s * b.x, c * a.y - s * b.y};
      tile[lj] = C2{s * a.x + c * b.x, s * a.y + c * b.y};
    }
  } else {
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const uint32_t li = li0 | insert_zero((uint32_t)(NT * j), pivot), lj = li ^ xl;
      const C2 cs = lut[code0 ^ d.jcode[j]];
      const R c = cs.x, s = sgn * cs.y;
      const C2 a = tile[li], b = tile[lj];
      tile[li] = C2{c * a.x + s * b.y, c * a.y - s * b.x};
      tile[lj] = C2{c * b.x + s * a.y, c * b.y - s * a.x};
    }
  }
}

template <typename R, bool STREAM, int P, bool GUARD>
__global__ void __launch_bounds__(NT, 4) k_sweep(R *psi, int n, PassDesc pd, const GroupDesc *groups,
                                                 const typename Vec2<R>::type *lut, int inverse) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(sizeof(C2), pd, 1, 0);
  const Tile<R> tc = stage_pass<R>(smem, pd, L, groups, lut);
  C2 *tile = reinterpret_cast<C2 *>(smem + L.tiles);
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const R sgn = inverse ? (R)-1 : (R)1;
  const int ng = pd.g_end - pd.g_begin;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(t, pd.umask);
    load_tile<R, STREAM>(psi, base, tc, reinterpret_cast<V *>(tile));
    __syncthreads();
    const uint64_t tpacked = t << pd.T;
    for (int k = 0; k < ng; ++k) {
      const int g = inverse ? ng - 1 - k : k;
      rot_group<R, P, GUARD>(tile, tc.gs[g], tc, tpacked, sgn);
      __syncthreads();
    }
    store_tile<R, STREAM>(psi, base, tc, reinterpret_cast<const V *>(tile));
    __syncthreads();
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

template <typename R, bool STREAM, int P, bool GUARD>
__global__ void __launch_bounds__(NT, 4) k_expect(const R *psi, int n, PassDesc pd,
                                                  const GroupDesc *groups,
                                                  const typename Vec2<R>::type *lut, double *partial,
                                                  int first_pass) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(sizeof(C2), pd, 1, sizeof(double) * (NT / 32));
  const Tile<R> tc = stage_pass<R>(smem, pd, L, groups, lut);
  C2 *tile = reinterpret_cast<C2 *>(smem + L.tiles);
  double *red = reinterpret_cast<double *>(smem + L.extra);
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const int ng = pd.g_end - pd.g_begin;
  const uint32_t tid = threadIdx.x;
  Kahan<R> acc_e, acc_n;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(t, pd.umask);
    load_tile<R, STREAM>(psi, base, tc, reinterpret_cast<V *>(tile));
    __syncthreads();
    const uint64_t tpacked = t << pd.T;
    if (first_pass) {
      R s = 0;
#pragma unroll
      for (int j = 0; j < 2 * P; ++j) {
        const uint32_t l = tid + NT * j;
        if (GUARD && l >= tc.amps) break;
        const C2 a = tile[l];
        s += a.x * a.x + a.y * a.y;
      }
      acc_n.add(s);
    }
    for (int k = 0; k < ng; ++k) {
      const GroupDesc &d = tc.gs[k];
      const C2 *lt = tc.lut + d.lut;
      const int r = d.r;
      R s = 0;
      if (d.kind == KIND_DIAG) {
        const uint32_t code0 = thread_code(d, r, tpacked | tid);
#pragma unroll
        for (int j = 0; j < 2 * P; ++j) {
          const uint32_t l = tid + NT * j;
          if (GUARD && l >= tc.amps) break;
          const R dv = lt[code0 ^ d.jcode[j]].x;
          const C2 a = tile[l];
          s += dv * (a.x * a.x + a.y * a.y);
        }
      } else if (!GUARD || tid < (tc.amps >> 1)) {
        const int pivot = d.pivot;
        const uint32_t xl = d.xl;
        const uint32_t li0 = insert_zero(tid, pivot);
        const uint32_t code0 = thread_code(d, r, tpacked | li0);
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const uint32_t li = li0 | insert_zero((uint32_t)(NT * j), pivot), lj = li ^ xl;
          const C2 rq = lt[code0 ^ d.jcode[j]];
          const C2 a = tile[li], b = tile[lj];
          // w = conj(a) b ; contribution 2 (R Re w + Q Im w)
          const R wr = a.x * b.x + a.y * b.y;
          const R wi = a.x * b.y - a.y * b.x;
          s += rq.x * wr + rq.y * wi;
        }
        s *= 2;
      }
      acc_e.add(s);
    }
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

// ------------------------------------------------------------------ H apply

template <typename R, bool STREAM, int P, bool GUARD>
__global__ void __launch_bounds__(NT, 3) k_happly(const R *psi, R *lam, int n, PassDesc pd,
                                                  const GroupDesc *groups,
                                                  const typename Vec2<R>::type *lut, int first_pass) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(sizeof(C2), pd, 2, 0);
  const Tile<R> tc = stage_pass<R>(smem, pd, L, groups, lut);
  C2 *tp = reinterpret_cast<C2 *>(smem + L.tiles);
  C2 *tl = tp + tc.amps;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const int ng = pd.g_end - pd.g_begin;
  const uint32_t tid = threadIdx.x;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(t, pd.umask);
    load_tile<R, STREAM>(psi, base, tc, reinterpret_cast<V *>(tp));
    if (first_pass) {
      for (uint32_t l = tid; l < tc.amps; l += NT) tl[l] = C2{0, 0};
    } else {
      load_tile<R, STREAM>(lam, base, tc, reinterpret_cast<V *>(tl));
    }
    __syncthreads();
    const uint64_t tpacked = t << pd.T;
    for (int k = 0; k < ng; ++k) {
      const GroupDesc &d = tc.gs[k];
      const C2 *lt = tc.lut + d.lut;
      const int r = d.r;
      if (d.kind == KIND_DIAG) {
        const uint32_t code0 = thread_code(d, r, tpacked | tid);
#pragma unroll
        for (int j = 0; j < 2 * P; ++j) {
          const uint32_t l = tid + NT * j;
          if (GUARD && l >= tc.amps) break;
          const R dv = lt[code0 ^ d.jcode[j]].x;
          const C2 a = tp[l];
          C2 o = tl[l];
          o.x += dv * a.x;
          o.y += dv * a.y;
          tl[l] = o;
        }
      } else if (!GUARD || tid < (tc.amps >> 1)) {
        const int pivot = d.pivot;
        const uint32_t xl = d.xl;
        const uint32_t li0 = insert_zero(tid, pivot);
        const uint32_t code0 = thread_code(d, r, tpacked | li0);
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const uint32_t li = li0 | insert_zero((uint32_t)(NT * j), pivot), lj = li ^ xl;
          const C2 rq = lt[code0 ^ d.jcode[j]];
          const C2 a = tp[li], b = tp[lj];
          C2 oi = tl[li], oj = tl[lj];
          // lam_i += (R - iQ) psi_j ; lam_j += (R + iQ) psi_i
          oi.x += rq.x * b.x + rq.y * b.y;
          oi.y += rq.x * b.y - rq.y * b.x;
          oj.x += rq.x * a.x - rq.y * a.y;
          oj.y += rq.x * a.y + rq.y * a.x;
          tl[li] = oi;
          tl[lj] = oj;
        }
      }
      __syncthreads();
    }
    store_tile<R, STREAM>(lam, base, tc, reinterpret_cast<const V *>(tl));
    __syncthreads();
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

template <typename R, bool STREAM, int P, bool GUARD>
__global__ void __launch_bounds__(NT, 2) k_reverse(R *psi, R *lam, int n, PassDesc pd,
                                                   const GroupDesc *groups,
                                                   const typename Vec2<R>::type *lut,
                                                   const uint64_t *signmask, double *partial) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L =
      smem_layout(sizeof(C2), pd, 2, sizeof(double) * RP_MAX + sizeof(R) * (NT / 32) * M_MAX);
  const Tile<R> tc = stage_pass<R>(smem, pd, L, groups, lut);
  C2 *tp = reinterpret_cast<C2 *>(smem + L.tiles);
  C2 *tl = tp + tc.amps;
  double *acc = reinterpret_cast<double *>(smem + L.extra);   // [RP_MAX]
  R *wpart = reinterpret_cast<R *>(acc + RP_MAX);             // [NT/32][M_MAX]
  const int nrot = pd.rot_end - pd.rot_begin;
  for (int k = threadIdx.x; k < nrot; k += NT) acc[k] = 0.0;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const int ng = pd.g_end - pd.g_begin;
  const uint32_t tid = threadIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(t, pd.umask);
    load_tile<R, STREAM>(psi, base, tc, reinterpret_cast<V *>(tp));
    load_tile<R, STREAM>(lam, base, tc, reinterpret_cast<V *>(tl));
    __syncthreads();
    const uint64_t tpacked = t << pd.T;
    for (int k = ng - 1; k >= 0; --k) {
      const GroupDesc &d = tc.gs[k];
      const C2 *lt = tc.lut + d.lut;
      const int kind = d.kind, r = d.r, m = d.m;
      const int rot0 = (int)d.rot0;
      const uint64_t *sm = signmask + pd.rot_begin + rot0;
      uint64_t mask[M_MAX];
      R a_k[M_MAX];
#pragma unroll
      for (int q = 0; q < M_MAX; ++q) {
        mask[q] = q < m ? __ldg(&sm[q]) : 0ull;
        a_k[q] = 0;
      }
      if (kind == KIND_DIAG) {
        const uint32_t code0 = thread_code(d, r, tpacked | tid);
#pragma unroll
        for (int j = 0; j < 2 * P; ++j) {
          const uint32_t l = tid + NT * j;
          if (GUARD && l >= tc.amps) break;
          const uint32_t code = code0 ^ d.jcode[j];
          const C2 cs = lt[code];
          const C2 a = tp[l], b = tl[l];
          const R val = b.x * a.y - b.y * a.x;   // Im(conj(lam) psi)
#pragma unroll
          for (int q = 0; q < M_MAX; ++q)
            if (q < m) a_k[q] += ((mask[q] >> code) & 1) ? -val : val;
          const R c = cs.x, s = -cs.y;
          tp[l] = C2{c * a.x + s * a.y, c * a.y - s * a.x};
          tl[l] = C2{c * b.x + s * b.y, c * b.y - s * b.x};
        }
      } else if (!GUARD || tid < (tc.amps >> 1)) {
        const int pivot = d.pivot;
        const uint32_t xl = d.xl;
        const uint32_t li0 = insert_zero(tid, pivot);
        const uint32_t code0 = thread_code(d, r, tpacked | li0);
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const uint32_t li = li0 | insert_zero((uint32_t)(NT * j), pivot), lj = li ^ xl;
          const uint32_t code = code0 ^ d.jcode[j];
          const C2 cs = lt[code];
          const C2 pa = tp[li], pb = tp[lj], la = tl[li], lb = tl[lj];
          R val;
          if (kind == KIND_REAL) {
            // Re(conj(lam_j) psi_i - conj(lam_i) psi_j)
            val = (lb.x * pa.x + lb.y * pa.y) - (la.x * pb.x + la.y * pb.y);
          } else {
            // Im(conj(lam_i) psi_j + conj(lam_j) psi_i)
            val = (la.x * pb.y - la.y * pb.x) + (lb.x * pa.y - lb.y * pa.x);
          }
#pragma unroll
          for (int q = 0; q < M_MAX; ++q)
            if (q < m) a_k[q] += ((mask[q] >> code) & 1) ? -val : val;
          const R c = cs.x, s = -cs.y;
          if (kind == KIND_REAL) {
            tp[li] = C2{c * pa.x - s * pb.x, c * pa.y - s * pb.y};
            tp[lj] = C2{s * pa.x + c * pb.x, s * pa.y + c * pb.y};
            tl[li] = C2{c * la.x - s * lb.x, c * la.y - s * lb.y};
            tl[lj] = C2{s * la.x + c * lb.x, s * la.y + c * lb.y};
          } else {
            tp[li] = C2{c * pa.x + s * pb.y, c * pa.y - s * pb.x};
            tp[lj] = C2{c * pb.x + s * pa.y, c * pb.y - s * pa.x};
            tl[li] = C2{c * la.x + s * lb.y, c * la.y - s * lb.x};
            tl[lj] = C2{c * lb.x + s * la.y, c * lb.y - s * la.x};
          }
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
    store_tile<R, STREAM>(psi, base, tc, reinterpret_cast<const V *>(tp));
    store_tile<R, STREAM>(lam, base, tc, reinterpret_cast<const V *>(tl));
    __syncthreads();
  }
  for (int k = threadIdx.x; k < nrot; k += NT) partial[(size_t)blockIdx.x * RP_MAX + k] = acc[k];
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

template <typename K>
cudaError_t prepare(K kernel, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

unsigned grid_for(uint64_t ntiles, int per_sm) {
  const uint64_t cap = (uint64_t)sm_count() * (uint64_t)per_sm;
  return (unsigned)(ntiles < cap ? ntiles : cap);
}

bool streaming(int n, int bytes) { return ((uint64_t)bytes << n) > (64ull << 20); }

// Pick the kernel instantiation for a pass: P = 2^(T-1) / NT pairs per thread.
#define Q2_DISPATCH(KERNEL, R, n, T, ...)                                              \
  [&]() -> decltype(&KERNEL<R, true, 1, true>) {                                     \
    const bool st_ = streaming(n, 2 * (int)sizeof(R));                               \
    switch (T) {                                                                       \
      case 9: return st_ ? &KERNEL<R, true, 1, false> : &KERNEL<R, false, 1, false>;  \
      case 10: return st_ ? &KERNEL<R, true, 2, false> : &KERNEL<R, false, 2, false>; \
      case 11: return st_ ? &KERNEL<R, true, 4, false> : &KERNEL<R, false, 4, false>; \
      case 12: return st_ ? &KERNEL<R, true, 8, false> : &KERNEL<R, false, 8, false>; \
      case 13: return st_ ? &KERNEL<R, true, 16, false> : &KERNEL<R, false, 16, false>; \
      default: return st_ ? &KERNEL<R, true, 1, true> : &KERNEL<R, false, 1, true>;   \
    }                                                                                  \
  }()

}  // namespace

size_t tile_smem_bytes(int amp_bytes, int T, int C, int vectors) {
  PassDesc pd{};
  pd.T = T;
  pd.C = C;
  pd.g_begin = 0;
  pd.g_end = G_STAGE;
  pd.lut_count = LUT_STAGE;
  return smem_layout(amp_bytes, pd, vectors, sizeof(double) * (NT / 32)).total;
}

size_t reverse_smem_bytes(int amp_bytes, int T, int C) {
  PassDesc pd{};
  pd.T = T;
  pd.C = C;
  pd.g_begin = 0;
  pd.g_end = G_STAGE;
  pd.lut_count = LUT_STAGE;
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
cudaError_t launch_sweep(R *psi, int n, const PassDesc &pd, const GroupDesc *groups, const void *lut,
                         bool inverse, cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  const size_t smem = smem_layout(sizeof(C2), pd, 1, 0).total;
  auto k = Q2_DISPATCH(k_sweep, R, n, pd.T);
  cudaError_t e = prepare(k, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = grid_for(1ull << (n - pd.T), blocks_per_sm(k, smem));
  k<<<grid, NT, smem, st>>>(psi, n, pd, groups, reinterpret_cast<const C2 *>(lut), inverse ? 1 : 0);
  return cudaGetLastError();
}

template <typename R>
int expect_grid(int n, int T, int C) {
  using C2 = typename Vec2<R>::type;
  const size_t smem = tile_smem_bytes(sizeof(C2), T, C, 1);
  auto k = Q2_DISPATCH(k_expect, R, n, T);
  prepare(k, smem);
  return (int)grid_for(1ull << (n - T), blocks_per_sm(k, smem));
}

template <typename R>
cudaError_t launch_expect(const R *psi, int n, const PassDesc &pd, const GroupDesc *groups,
                          const void *lut, double *partial, int grid, bool first, cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  const size_t smem = smem_layout(sizeof(C2), pd, 1, sizeof(double) * (NT / 32)).total;
  auto k = Q2_DISPATCH(k_expect, R, n, pd.T);
  cudaError_t e = prepare(k, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, NT, smem, st>>>(psi, n, pd, groups, reinterpret_cast<const C2 *>(lut), partial, first ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_reduce_pairs(const double *partial, int nblocks, double *out, cudaStream_t st) {
  k_reduce_pairs<<<1, NT, 0, st>>>(partial, nblocks, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_happly(const R *psi, R *lam, int n, const PassDesc &pd, const GroupDesc *groups,
                          const void *lut, bool first, cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  const size_t smem = smem_layout(sizeof(C2), pd, 2, 0).total;
  auto k = Q2_DISPATCH(k_happly, R, n, pd.T);
  cudaError_t e = prepare(k, smem);
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
int reverse_grid(int n, int T, int C) {
  using C2 = typename Vec2<R>::type;
  const size_t smem = reverse_smem_bytes(sizeof(C2), T, C);
  auto k = Q2_DISPATCH(k_reverse, R, n, T);
  prepare(k, smem);
  return (int)grid_for(1ull << (n - T), blocks_per_sm(k, smem));
}

template <typename R>
cudaError_t launch_reverse(R *psi, R *lam, int n, const PassDesc &pd, const GroupDesc *groups,
                           const void *lut, const uint64_t *signmask, double *partial, double *gphi,
                           cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  const size_t smem =
      smem_layout(sizeof(C2), pd, 2, sizeof(double) * RP_MAX + sizeof(R) * (NT / 32) * M_MAX).total;
  auto k = Q2_DISPATCH(k_reverse, R, n, pd.T);
  cudaError_t e = prepare(k, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = grid_for(1ull << (n - pd.T), blocks_per_sm(k, smem));
  k<<<grid, NT, smem, st>>>(psi, lam, n, pd, groups, reinterpret_cast<const C2 *>(lut), signmask, partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nrot = pd.rot_end - pd.rot_begin;
  k_reduce_rot<<<(nrot + 127) / 128, 128, 0, st>>>(partial, (int)grid, nrot, gphi + pd.rot_begin);
  return cudaGetLastError();
}

#define Q2_INST(R)                                                                                  \
  template cudaError_t launch_init_hf<R>(R *, int, int, cudaStream_t);                             \
  template cudaError_t launch_sweep<R>(R *, int, const PassDesc &, const GroupDesc *, const void *, \
                                       bool, cudaStream_t);                                         \
  template int expect_grid<R>(int, int, int);                                                       \
  template cudaError_t launch_expect<R>(const R *, int, const PassDesc &, const GroupDesc *,        \
                                        const void *, double *, int, bool, cudaStream_t);           \
  template cudaError_t launch_happly<R>(const R *, R *, int, const PassDesc &, const GroupDesc *,   \
                                        const void *, bool, cudaStream_t);                          \
  template int dot_grid<R>(int);                                                                    \
  template cudaError_t launch_dot<R>(const R *, const R *, int, double *, int, cudaStream_t);       \
  template int reverse_grid<R>(int, int, int);                                                      \
  template cudaError_t launch_reverse<R>(R *, R *, int, const PassDesc &, const GroupDesc *,        \
                                         const void *, const uint64_t *, double *, double *,        \
                                         cudaStream_t);

Q2_INST(float)
Q2_INST(double)

}  // namespace q2
