// Tile kernels of the state-vector engine (sm_103a).
//
// Every kernel here is HBM-streaming: a persistent grid walks the 2^(n-T)
// tiles of one pass; each CTA gathers a tile (2^(T-C) chunks of 2^C
// contiguous amplitudes) into shared memory with 16-byte loads, applies all
// groups of the pass there, and writes the tile back (or only reduces it).
// Tiles are cosets of the pass's local subspace W (see q2_internal.h), so a
// pass touches every amplitude exactly once and tiles never overlap.
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

// Tile geometry shared by all tile kernels.
struct TileCtx {
  int T, C;
  uint32_t tile_amps;     // 2^T
  uint64_t *off;          // smem: 2^(T-C) chunk offsets
};

__device__ __forceinline__ void build_offsets(const PassDesc &pd, uint64_t *off) {
  const int nh = 1 << (pd.T - pd.C);
  for (int h = threadIdx.x; h < nh; h += blockDim.x) {
    uint64_t o = 0;
    for (int b = 0; b < pd.T - pd.C; ++b)
      if ((h >> b) & 1) o ^= pd.w[pd.C + b];
    off[h] = o;
  }
}

__device__ __forceinline__ uint64_t tile_base(uint64_t t, uint64_t umask) {
  return deposit_bits(t, umask);
}

// Amplitude index of vector v (16-byte unit) of a tile.
template <typename R>
__device__ __forceinline__ uint64_t vec_index(uint64_t base, uint32_t v, const TileCtx &tc) {
  const uint32_t l = v * Vec16<R>::amps;
  const uint32_t cm = (1u << tc.C) - 1u;
  return (base ^ tc.off[l >> tc.C]) | (l & cm);
}

// Gather one tile of `src` into shared memory.
template <typename R, bool STREAM>
__device__ __forceinline__ void load_tile(const R *src, uint64_t base, const TileCtx &tc,
                                          typename Vec16<R>::type *dst) {
  using V = typename Vec16<R>::type;
  const uint32_t nv = tc.tile_amps / Vec16<R>::amps;
  const V *g = reinterpret_cast<const V *>(src);
  for (uint32_t v0 = 0; v0 < nv; v0 += 8 * NT) {
    V buf[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t v = v0 + k * NT + threadIdx.x;
      if (v < nv) buf[k] = ld16<V, STREAM>(g + vec_index<R>(base, v, tc) / Vec16<R>::amps);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t v = v0 + k * NT + threadIdx.x;
      if (v < nv) dst[v] = buf[k];
    }
  }
}

template <typename R, bool STREAM>
__device__ __forceinline__ void store_tile(R *dstg, uint64_t base, const TileCtx &tc,
                                           const typename Vec16<R>::type *src) {
  using V = typename Vec16<R>::type;
  const uint32_t nv = tc.tile_amps / Vec16<R>::amps;
  V *g = reinterpret_cast<V *>(dstg);
  for (uint32_t v = threadIdx.x; v < nv; v += NT)
    st16<V, STREAM>(g + vec_index<R>(base, v, tc) / Vec16<R>::amps, src[v]);
}

// Code of the thread's first element of a group in the current tile.
__device__ __forceinline__ uint32_t thread_code(const GroupDesc *gd, int r, uint64_t packed) {
  uint32_t code = 0;
  for (int l = 0; l < r; ++l) code |= (uint32_t)par64(packed & __ldg(&gd->bp[l])) << l;
  return code;
}

__device__ __forceinline__ uint32_t jcode_of(const GroupDesc *gd, int j) {
  return __ldg(&gd->jcode[j]);
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

// ------------------------------------------------------------------ rotation sweep

// Apply rotation group gd (sign +1 forward, -1 inverse) to a shared-memory tile.
template <typename R>
__device__ __forceinline__ void rot_group(typename Vec2<R>::type *tile, const GroupDesc *gd,
                                          const typename Vec2<R>::type *lut, uint64_t tpacked,
                                          int T, R sgn) {
  using C2 = typename Vec2<R>::type;
  const int kind = __ldg(&gd->kind);
  const int r = __ldg(&gd->r);
  const uint32_t lut0 = __ldg(&gd->lut);
  if (kind == KIND_DIAG) {
    const uint32_t n_amp = 1u << T;
    const int P = n_amp > NT ? (int)(n_amp / NT) : 1;
    const uint32_t code0 = thread_code(gd, r, tpacked | threadIdx.x);
    for (int j = 0; j < P; ++j) {
      const uint32_t l = threadIdx.x + NT * j;
      if (l >= n_amp) break;
      const C2 cs = __ldg(&lut[lut0 + (code0 ^ jcode_of(gd, j))]);
      const R c = cs.x, s = sgn * cs.y;
      const C2 a = tile[l];
      tile[l] = C2{c * a.x + s * a.y, c * a.y - s * a.x};
    }
    return;
  }
  const int pivot = __ldg(&gd->pivot);
  const uint32_t xl = __ldg(&gd->xl);
  const uint32_t n_pair = 1u << (T - 1);
  const int P = n_pair > NT ? (int)(n_pair / NT) : 1;
  const uint32_t code0 = thread_code(gd, r, tpacked | insert_zero(threadIdx.x, pivot));
  if (kind == KIND_REAL) {
#pragma unroll 4
    for (int j = 0; j < P; ++j) {
      const uint32_t q = threadIdx.x + NT * j;
      if (q >= n_pair) break;
      const uint32_t li = insert_zero(q, pivot), lj = li ^ xl;
      const C2 cs = __ldg(&lut[lut0 + (code0 ^ jcode_of(gd, j))]);
      const R c = cs.x, s = sgn * cs.y;
      const C2 a = tile[li], b = tile[lj];
      tile[li] = C2{c * a.x - s * b.x, c * a.y - s * b.y};
      tile[lj] = C2{s * a.x + c * b.x, s * a.y + c * b.y};
    }
  } else {
#pragma unroll 4
    for (int j = 0; j < P; ++j) {
      const uint32_t q = threadIdx.x + NT * j;
      if (q >= n_pair) break;
      const uint32_t li = insert_zero(q, pivot), lj = li ^ xl;
      const C2 cs = __ldg(&lut[lut0 + (code0 ^ jcode_of(gd, j))]);
      const R c = cs.x, s = sgn * cs.y;
      const C2 a = tile[li], b = tile[lj];
      tile[li] = C2{c * a.x + s * b.y, c * a.y - s * b.x};
      tile[lj] = C2{c * b.x + s * a.y, c * b.y - s * a.x};
    }
  }
}

template <typename R, bool STREAM>
__global__ void __launch_bounds__(NT) k_sweep(R *psi, int n, PassDesc pd, const GroupDesc *groups,
                                              const typename Vec2<R>::type *lut, int inverse) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  TileCtx tc;
  tc.T = pd.T;
  tc.C = pd.C;
  tc.tile_amps = 1u << pd.T;
  C2 *tile = reinterpret_cast<C2 *>(smem);
  tc.off = reinterpret_cast<uint64_t *>(smem + sizeof(C2) * tc.tile_amps);
  build_offsets(pd, tc.off);
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const R sgn = inverse ? (R)-1 : (R)1;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(t, pd.umask);
    load_tile<R, STREAM>(psi, base, tc, reinterpret_cast<V *>(tile));
    __syncthreads();
    const uint64_t tpacked = t << pd.T;
    if (!inverse) {
      for (int g = pd.g_begin; g < pd.g_end; ++g) {
        rot_group<R>(tile, groups + g, lut, tpacked, pd.T, sgn);
        __syncthreads();
      }
    } else {
      for (int g = pd.g_end - 1; g >= pd.g_begin; --g) {
        rot_group<R>(tile, groups + g, lut, tpacked, pd.T, sgn);
        __syncthreads();
      }
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

template <typename R, bool STREAM>
__global__ void __launch_bounds__(NT) k_expect(const R *psi, int n, PassDesc pd,
                                               const GroupDesc *groups,
                                               const typename Vec2<R>::type *lut, double *partial,
                                               int first_pass) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  TileCtx tc;
  tc.T = pd.T;
  tc.C = pd.C;
  tc.tile_amps = 1u << pd.T;
  C2 *tile = reinterpret_cast<C2 *>(smem);
  tc.off = reinterpret_cast<uint64_t *>(smem + sizeof(C2) * tc.tile_amps);
  double *red = reinterpret_cast<double *>(tc.off + (1u << (pd.T - pd.C)));
  build_offsets(pd, tc.off);
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  Kahan<R> acc_e, acc_n;
  const uint32_t n_amp = tc.tile_amps, n_pair = n_amp >> 1;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(t, pd.umask);
    load_tile<R, STREAM>(psi, base, tc, reinterpret_cast<V *>(tile));
    __syncthreads();
    const uint64_t tpacked = t << pd.T;
    if (first_pass) {
      R s = 0;
      for (uint32_t l = threadIdx.x; l < n_amp; l += NT) {
        const C2 a = tile[l];
        s += a.x * a.x + a.y * a.y;
      }
      acc_n.add(s);
    }
    for (int g = pd.g_begin; g < pd.g_end; ++g) {
      const GroupDesc *gd = groups + g;
      const int kind = __ldg(&gd->kind), r = __ldg(&gd->r);
      const uint32_t lut0 = __ldg(&gd->lut);
      R s = 0;
      if (kind == KIND_DIAG) {
        const int P = n_amp > NT ? (int)(n_amp / NT) : 1;
        const uint32_t code0 = thread_code(gd, r, tpacked | threadIdx.x);
        for (int j = 0; j < P; ++j) {
          const uint32_t l = threadIdx.x + NT * j;
          if (l >= n_amp) break;
          const R d = __ldg(&lut[lut0 + (code0 ^ jcode_of(gd, j))]).x;
          const C2 a = tile[l];
          s += d * (a.x * a.x + a.y * a.y);
        }
      } else {
        const int pivot = __ldg(&gd->pivot);
        const uint32_t xl = __ldg(&gd->xl);
        const int P = n_pair > NT ? (int)(n_pair / NT) : 1;
        const uint32_t code0 = thread_code(gd, r, tpacked | insert_zero(threadIdx.x, pivot));
#pragma unroll 4
        for (int j = 0; j < P; ++j) {
          const uint32_t q = threadIdx.x + NT * j;
          if (q >= n_pair) break;
          const uint32_t li = insert_zero(q, pivot), lj = li ^ xl;
          const C2 rq = __ldg(&lut[lut0 + (code0 ^ jcode_of(gd, j))]);
          const C2 a = tile[li], b = tile[lj];
          // w = conj(a) b ; contribution 2 (R Re w + Q Im w)
          const R wr = a.x * b.x + a.y * b.y;
          const R wi = a.x * b.y - a.y * b.x;
          s += 2 * (rq.x * wr + rq.y * wi);
        }
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

template <typename R, bool STREAM>
__global__ void __launch_bounds__(NT) k_happly(const R *psi, R *lam, int n, PassDesc pd,
                                               const GroupDesc *groups,
                                               const typename Vec2<R>::type *lut, int first_pass) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  TileCtx tc;
  tc.T = pd.T;
  tc.C = pd.C;
  tc.tile_amps = 1u << pd.T;
  C2 *tp = reinterpret_cast<C2 *>(smem);
  C2 *tl = tp + tc.tile_amps;
  tc.off = reinterpret_cast<uint64_t *>(tl + tc.tile_amps);
  build_offsets(pd, tc.off);
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const uint32_t n_amp = tc.tile_amps, n_pair = n_amp >> 1;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(t, pd.umask);
    load_tile<R, STREAM>(psi, base, tc, reinterpret_cast<V *>(tp));
    if (first_pass) {
      for (uint32_t l = threadIdx.x; l < n_amp; l += NT) tl[l] = C2{0, 0};
    } else {
      load_tile<R, STREAM>(lam, base, tc, reinterpret_cast<V *>(tl));
    }
    __syncthreads();
    const uint64_t tpacked = t << pd.T;
    for (int g = pd.g_begin; g < pd.g_end; ++g) {
      const GroupDesc *gd = groups + g;
      const int kind = __ldg(&gd->kind), r = __ldg(&gd->r);
      const uint32_t lut0 = __ldg(&gd->lut);
      if (kind == KIND_DIAG) {
        const int P = n_amp > NT ? (int)(n_amp / NT) : 1;
        const uint32_t code0 = thread_code(gd, r, tpacked | threadIdx.x);
        for (int j = 0; j < P; ++j) {
          const uint32_t l = threadIdx.x + NT * j;
          if (l >= n_amp) break;
          const R d = __ldg(&lut[lut0 + (code0 ^ jcode_of(gd, j))]).x;
          const C2 a = tp[l];
          C2 o = tl[l];
          o.x += d * a.x;
          o.y += d * a.y;
          tl[l] = o;
        }
      } else {
        const int pivot = __ldg(&gd->pivot);
        const uint32_t xl = __ldg(&gd->xl);
        const int P = n_pair > NT ? (int)(n_pair / NT) : 1;
        const uint32_t code0 = thread_code(gd, r, tpacked | insert_zero(threadIdx.x, pivot));
#pragma unroll 4
        for (int j = 0; j < P; ++j) {
          const uint32_t q = threadIdx.x + NT * j;
          if (q >= n_pair) break;
          const uint32_t li = insert_zero(q, pivot), lj = li ^ xl;
          const C2 rq = __ldg(&lut[lut0 + (code0 ^ jcode_of(gd, j))]);
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

template <typename R, bool STREAM>
__global__ void __launch_bounds__(NT) k_reverse(R *psi, R *lam, int n, PassDesc pd,
                                                const GroupDesc *groups,
                                                const typename Vec2<R>::type *lut,
                                                const uint64_t *signmask, double *partial) {
  using C2 = typename Vec2<R>::type;
  using V = typename Vec16<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  TileCtx tc;
  tc.T = pd.T;
  tc.C = pd.C;
  tc.tile_amps = 1u << pd.T;
  C2 *tp = reinterpret_cast<C2 *>(smem);
  C2 *tl = tp + tc.tile_amps;
  tc.off = reinterpret_cast<uint64_t *>(tl + tc.tile_amps);
  double *acc = reinterpret_cast<double *>(tc.off + (1u << (pd.T - pd.C)));  // [RP_MAX]
  R *wpart = reinterpret_cast<R *>(acc + RP_MAX);                              // [NT/32][M_MAX]
  build_offsets(pd, tc.off);
  const int nrot = pd.rot_end - pd.rot_begin;
  for (int k = threadIdx.x; k < nrot; k += NT) acc[k] = 0.0;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pd.T);
  const uint32_t n_amp = tc.tile_amps, n_pair = n_amp >> 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(t, pd.umask);
    load_tile<R, STREAM>(psi, base, tc, reinterpret_cast<V *>(tp));
    load_tile<R, STREAM>(lam, base, tc, reinterpret_cast<V *>(tl));
    __syncthreads();
    const uint64_t tpacked = t << pd.T;
    for (int g = pd.g_end - 1; g >= pd.g_begin; --g) {
      const GroupDesc *gd = groups + g;
      const int kind = __ldg(&gd->kind), r = __ldg(&gd->r), m = __ldg(&gd->m);
      const uint32_t lut0 = __ldg(&gd->lut);
      const int rot0 = (int)__ldg(&gd->rot0);
      const uint64_t *sm = signmask + pd.rot_begin + rot0;
      uint64_t mask[M_MAX];
      R a_k[M_MAX];
#pragma unroll
      for (int k = 0; k < M_MAX; ++k) {
        mask[k] = k < m ? __ldg(&sm[k]) : 0ull;
        a_k[k] = 0;
      }
      if (kind == KIND_DIAG) {
        const int P = n_amp > NT ? (int)(n_amp / NT) : 1;
        const uint32_t code0 = thread_code(gd, r, tpacked | threadIdx.x);
        for (int j = 0; j < P; ++j) {
          const uint32_t l = threadIdx.x + NT * j;
          if (l >= n_amp) break;
          const uint32_t code = code0 ^ jcode_of(gd, j);
          const C2 cs = __ldg(&lut[lut0 + code]);
          const C2 a = tp[l], b = tl[l];
          const R val = b.x * a.y - b.y * a.x;   // Im(conj(lam) psi)
#pragma unroll
          for (int k = 0; k < M_MAX; ++k)
            if (k < m) a_k[k] += ((mask[k] >> code) & 1) ? -val : val;
          const R c = cs.x, s = -cs.y;
          tp[l] = C2{c * a.x + s * a.y, c * a.y - s * a.x};
          tl[l] = C2{c * b.x + s * b.y, c * b.y - s * b.x};
        }
      } else {
        const int pivot = __ldg(&gd->pivot);
        const uint32_t xl = __ldg(&gd->xl);
        const int P = n_pair > NT ? (int)(n_pair / NT) : 1;
        const uint32_t code0 = thread_code(gd, r, tpacked | insert_zero(threadIdx.x, pivot));
        for (int j = 0; j < P; ++j) {
          const uint32_t q = threadIdx.x + NT * j;
          if (q >= n_pair) break;
          const uint32_t li = insert_zero(q, pivot), lj = li ^ xl;
          const uint32_t code = code0 ^ jcode_of(gd, j);
          const C2 cs = __ldg(&lut[lut0 + code]);
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
          for (int k = 0; k < M_MAX; ++k)
            if (k < m) a_k[k] += ((mask[k] >> code) & 1) ? -val : val;
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
      for (int k = 0; k < M_MAX; ++k) {
        if (k < m) {
          R v = a_k[k];
          for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
          if (lane == 0) wpart[warp * M_MAX + k] = v;
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

template <typename K>
int blocks_per_sm(K kernel, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, NT, smem) != cudaSuccess) return 1;
  return b > 0 ? b : 1;
}

int sm_count() {
  static int cached = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  static int cached_dev = -1;
  if (cached < 0 || cached_dev != dev) {
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    cached_dev = dev;
  }
  return cached;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

uint64_t grid_for(uint64_t ntiles, int per_sm) {
  const uint64_t cap = (uint64_t)sm_count() * (uint64_t)per_sm;
  return ntiles < cap ? ntiles : cap;
}

}  // namespace

size_t tile_smem_bytes(int dtype_bytes, int T, int C, int vectors) {
  return (size_t)dtype_bytes * ((size_t)1 << T) * vectors + sizeof(uint64_t) * ((size_t)1 << (T - C)) +
         sizeof(double) * 64;
}

size_t reverse_smem_bytes(int dtype_bytes, int T, int C) {
  return tile_smem_bytes(dtype_bytes, T, C, 2) + sizeof(double) * RP_MAX +
         (size_t)(dtype_bytes / 2) * (NT / 32) * M_MAX;
}

int max_grid_blocks(int dtype_bytes, int T) {
  // upper bound on any tile kernel's grid (for partial buffers)
  (void)dtype_bytes;
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

static bool streaming(int n, int bytes) { return ((uint64_t)bytes << n) > (64ull << 20); }

template <typename R>
cudaError_t launch_sweep(R *psi, int n, const PassDesc &pd, const GroupDesc *groups,
                         const void *lut, bool inverse, cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  const size_t smem = tile_smem_bytes(sizeof(C2), pd.T, pd.C, 1);
  const uint64_t ntiles = 1ull << (n - pd.T);
  cudaError_t e;
  if (streaming(n, sizeof(C2))) {
    auto k = k_sweep<R, true>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)grid_for(ntiles, blocks_per_sm(k, smem));
    k<<<grid, NT, smem, st>>>(psi, n, pd, groups, reinterpret_cast<const C2 *>(lut), inverse ? 1 : 0);
  } else {
    auto k = k_sweep<R, false>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)grid_for(ntiles, blocks_per_sm(k, smem));
    k<<<grid, NT, smem, st>>>(psi, n, pd, groups, reinterpret_cast<const C2 *>(lut), inverse ? 1 : 0);
  }
  return cudaGetLastError();
}

template <typename R>
int expect_grid(int n, int T, int C) {
  using C2 = typename Vec2<R>::type;
  const size_t smem = tile_smem_bytes(sizeof(C2), T, C, 1);
  const uint64_t ntiles = 1ull << (n - T);
  auto k = streaming(n, sizeof(C2)) ? k_expect<R, true> : k_expect<R, false>;
  set_smem(k, smem);
  return (int)grid_for(ntiles, blocks_per_sm(k, smem));
}

template <typename R>
cudaError_t launch_expect(const R *psi, int n, const PassDesc &pd, const GroupDesc *groups,
                          const void *lut, double *partial, int grid, bool first, cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  const size_t smem = tile_smem_bytes(sizeof(C2), pd.T, pd.C, 1);
  cudaError_t e;
  if (streaming(n, sizeof(C2))) {
    auto k = k_expect<R, true>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    k<<<grid, NT, smem, st>>>(psi, n, pd, groups, reinterpret_cast<const C2 *>(lut), partial, first);
  } else {
    auto k = k_expect<R, false>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    k<<<grid, NT, smem, st>>>(psi, n, pd, groups, reinterpret_cast<const C2 *>(lut), partial, first);
  }
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
  const size_t smem = tile_smem_bytes(sizeof(C2), pd.T, pd.C, 2);
  const uint64_t ntiles = 1ull << (n - pd.T);
  cudaError_t e;
  if (streaming(n, sizeof(C2))) {
    auto k = k_happly<R, true>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)grid_for(ntiles, blocks_per_sm(k, smem));
    k<<<grid, NT, smem, st>>>(psi, lam, n, pd, groups, reinterpret_cast<const C2 *>(lut), first);
  } else {
    auto k = k_happly<R, false>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    const unsigned grid = (unsigned)grid_for(ntiles, blocks_per_sm(k, smem));
    k<<<grid, NT, smem, st>>>(psi, lam, n, pd, groups, reinterpret_cast<const C2 *>(lut), first);
  }
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
  const uint64_t ntiles = 1ull << (n - T);
  auto k = streaming(n, sizeof(C2)) ? k_reverse<R, true> : k_reverse<R, false>;
  set_smem(k, smem);
  return (int)grid_for(ntiles, blocks_per_sm(k, smem));
}

template <typename R>
cudaError_t launch_reverse(R *psi, R *lam, int n, const PassDesc &pd, const GroupDesc *groups,
                           const void *lut, const uint64_t *signmask, double *partial, double *gphi,
                           cudaStream_t st) {
  using C2 = typename Vec2<R>::type;
  const size_t smem = reverse_smem_bytes(sizeof(C2), pd.T, pd.C);
  const uint64_t ntiles = 1ull << (n - pd.T);
  cudaError_t e;
  unsigned grid;
  if (streaming(n, sizeof(C2))) {
    auto k = k_reverse<R, true>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    grid = (unsigned)grid_for(ntiles, blocks_per_sm(k, smem));
    k<<<grid, NT, smem, st>>>(psi, lam, n, pd, groups, reinterpret_cast<const C2 *>(lut), signmask,
                              partial);
  } else {
    auto k = k_reverse<R, false>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    grid = (unsigned)grid_for(ntiles, blocks_per_sm(k, smem));
    k<<<grid, NT, smem, st>>>(psi, lam, n, pd, groups, reinterpret_cast<const C2 *>(lut), signmask,
                              partial);
  }
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
