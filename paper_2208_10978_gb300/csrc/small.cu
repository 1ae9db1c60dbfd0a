// Batched small-state kernel (serving path).
//
// One persistent launch evaluates a whole batch of small problems: CTA b
// takes requests b, b + gridDim, ...; for each it keeps psi (and lambda when
// the gradient is wanted) for all 2^n <= 4096 amplitudes in shared memory and
// runs, without touching HBM except for its tables:
//   HF determinant (Eq. jw-wfn-map) -> every rotation group in order (product
//   formula after Eq. ucc) -> energy sum_t c_t <P_t> and <psi|psi>
//   (Eq. qubit-ham-detail), or lambda = H psi, E = Re<psi|lambda> and the
//   reverse loop of Algorithm 1 with dE/dphi_k = Im<lambda|P_k|psi>.
// Plans use the identity local basis (one tile = the whole state), so a
// group's xmask and code basis are plain global masks and codes are parities
// of the amplitude index.  Reductions are fixed-order per CTA, so a request's
// result does not depend on the rest of the batch.
#include <cuda_runtime.h>

#include <mutex>
#include <set>

#include "small.h"

namespace q2 {

template <typename R> struct SVec2;
template <> struct SVec2<float> { using type = float2; };
template <> struct SVec2<double> { using type = double2; };

__device__ __forceinline__ uint32_t code_of(const GroupDesc &g, int r, uint32_t i) {
  uint32_t c = 0;
  for (int l = 0; l < r; ++l) c |= (uint32_t)(__popc(i & (uint32_t)g.bp[l]) & 1) << l;
  return c;
}

template <typename C2, typename R>
__device__ __forceinline__ void srot_real(C2 &a, C2 &b, R c, R s) {
  const C2 x = a, y = b;
  a = C2{c * x.x - s * y.x, c * x.y - s * y.y};
  b = C2{s * x.x + c * y.x, s * x.y + c * y.y};
}
template <typename C2, typename R>
__device__ __forceinline__ void srot_xrot(C2 &a, C2 &b, R c, R s) {
  const C2 x = a, y = b;
  a = C2{c * x.x + s * y.y, c * x.y - s * y.x};
  b = C2{c * y.x + s * x.y, c * y.y - s * x.x};
}
template <typename C2, typename R>
__device__ __forceinline__ void sphase(C2 &a, R c, R s) {
  const C2 x = a;
  a = C2{c * x.x + s * x.y, c * x.y - s * x.x};
}

// Apply (sgn = +1) or undo (sgn = -1) one rotation group on a state in shared memory.
template <typename R>
__device__ void small_rot(typename SVec2<R>::type *psi, uint32_t dim, const GroupDesc &g,
                          const typename SVec2<R>::type *lut, R sgn) {
  using C2 = typename SVec2<R>::type;
  const int r = g.r;
  const C2 *L = lut + g.lut;
  if (g.kind == KIND_DIAG) {
    for (uint32_t i = threadIdx.x; i < dim; i += blockDim.x) {
      const C2 cs = L[code_of(g, r, i)];
      sphase(psi[i], cs.x, sgn * cs.y);
    }
    return;
  }
  const int pivot = g.pivot;
  const uint32_t x = g.xl;
  const bool real = g.kind == KIND_REAL;
  for (uint32_t q = threadIdx.x; q < (dim >> 1); q += blockDim.x) {
    const uint32_t i = insert_zero(q, pivot), j = i ^ x;
    const C2 cs = L[code_of(g, r, i)];
    C2 a = psi[i], b = psi[j];
    if (real) srot_real(a, b, cs.x, sgn * cs.y);
    else srot_xrot(a, b, cs.x, sgn * cs.y);
    psi[i] = a;
    psi[j] = b;
  }
}

__device__ __forceinline__ double sblock_sum(double v, double *scratch) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += scratch[w];
  __syncthreads();
  return s;
}

template <typename R>
__global__ void __launch_bounds__(NT) k_batch(const BatchItem *items, int n_items) {
  using C2 = typename SVec2<R>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[NT / 32];
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const BatchItem B = items[it];
    const uint32_t dim = 1u << B.n;
    C2 *psi = reinterpret_cast<C2 *>(smem);
    C2 *lam = psi + dim;
    const C2 *rl = static_cast<const C2 *>(B.rlut);
    const C2 *hl = static_cast<const C2 *>(B.hlut);
    const uint32_t hf = (1u << B.n_elec) - 1u;
    for (uint32_t i = threadIdx.x; i < dim; i += NT) psi[i] = C2{(R)(i == hf ? 1 : 0), (R)0};
    __syncthreads();
    for (int g = 0; g < B.nrg; ++g) {
      small_rot<R>(psi, dim, B.rg[g], rl, (R)1);
      __syncthreads();
    }
    double e_raw = 0.0, nrm = 0.0;
    if (!B.want_grad) {
      double acc = 0.0, an = 0.0;
      for (uint32_t i = threadIdx.x; i < dim; i += NT) an += (double)(psi[i].x * psi[i].x + psi[i].y * psi[i].y);
      for (int g = 0; g < B.nhg; ++g) {
        const GroupDesc &G = B.hg[g];
        const C2 *L = hl + G.lut;
        const int r = G.r;
        if (G.kind == KIND_DIAG) {
          for (uint32_t i = threadIdx.x; i < dim; i += NT) {
            const R d = L[code_of(G, r, i)].x;
            acc += (double)(d * (psi[i].x * psi[i].x + psi[i].y * psi[i].y));
          }
        } else {
          for (uint32_t q = threadIdx.x; q < (dim >> 1); q += NT) {
            const uint32_t i = insert_zero(q, G.pivot), j = i ^ G.xl;
            const C2 rq = L[code_of(G, r, i)];
            const C2 a = psi[i], b = psi[j];
            acc += 2.0 * (double)(rq.x * (a.x * b.x + a.y * b.y) + rq.y * (a.x * b.y - a.y * b.x));
          }
        }
      }
      e_raw = sblock_sum(acc, red);
      nrm = sblock_sum(an, red);
      if (threadIdx.x == 0) {
        B.out[0] = e_raw;
        B.out[1] = nrm;
      }
      __syncthreads();
      continue;
    }
    // lambda = H psi
    for (uint32_t i = threadIdx.x; i < dim; i += NT) lam[i] = C2{0, 0};
    __syncthreads();
    for (int g = 0; g < B.nhg; ++g) {
      const GroupDesc &G = B.hg[g];
      const C2 *L = hl + G.lut;
      const int r = G.r;
      if (G.kind == KIND_DIAG) {
        for (uint32_t i = threadIdx.x; i < dim; i += NT) {
          const R d = L[code_of(G, r, i)].x;
          lam[i].x += d * psi[i].x;
          lam[i].y += d * psi[i].y;
        }
      } else {
        for (uint32_t q = threadIdx.x; q < (dim >> 1); q += NT) {
          const uint32_t i = insert_zero(q, G.pivot), j = i ^ G.xl;
          const C2 rq = L[code_of(G, r, i)];
          const C2 a = psi[i], b = psi[j];
          lam[i].x += rq.x * b.x + rq.y * b.y;
          lam[i].y += rq.x * b.y - rq.y * b.x;
          lam[j].x += rq.x * a.x - rq.y * a.y;
          lam[j].y += rq.x * a.y + rq.y * a.x;
        }
      }
      __syncthreads();
    }
    {
      double ae = 0.0, an = 0.0;
      for (uint32_t i = threadIdx.x; i < dim; i += NT) {
        ae += (double)(psi[i].x * lam[i].x + psi[i].y * lam[i].y);
        an += (double)(psi[i].x * psi[i].x + psi[i].y * psi[i].y);
      }
      e_raw = sblock_sum(ae, red);
      nrm = sblock_sum(an, red);
      if (threadIdx.x == 0) {
        B.out[0] = e_raw;
        B.out[1] = nrm;
      }
    }
    // reverse sweep: per-rotation Im<lam|P_k|psi> at the state after the group, then undo it
    for (int g = B.nrg - 1; g >= 0; --g) {
      const GroupDesc &G = B.rg[g];
      const C2 *L = rl + G.lut;
      const int r = G.r, m = G.m;
      const int k0 = B.grot[g];
      double acc[M_MAX];
      uint64_t mk[M_MAX];
#pragma unroll
      for (int k = 0; k < M_MAX; ++k) {
        acc[k] = 0.0;
        mk[k] = k < m ? B.sm[k0 + k] : 0ull;
      }
      if (G.kind == KIND_DIAG) {
        for (uint32_t i = threadIdx.x; i < dim; i += NT) {
          const uint32_t code = code_of(G, r, i);
          const double val = (double)(lam[i].x * psi[i].y - lam[i].y * psi[i].x);
#pragma unroll
          for (int k = 0; k < M_MAX; ++k)
            if (k < m) acc[k] += ((mk[k] >> code) & 1) ? -val : val;
        }
      } else {
        for (uint32_t q = threadIdx.x; q < (dim >> 1); q += NT) {
          const uint32_t i = insert_zero(q, G.pivot), j = i ^ G.xl;
          const uint32_t code = code_of(G, r, i);
          const C2 pa = psi[i], pb = psi[j], la = lam[i], lb = lam[j];
          double val;
          if (G.kind == KIND_REAL)
            val = (double)((lb.x * pa.x + lb.y * pa.y) - (la.x * pb.x + la.y * pb.y));
          else
            val = (double)((la.x * pb.y - la.y * pb.x) + (lb.x * pa.y - lb.y * pa.x));
#pragma unroll
          for (int k = 0; k < M_MAX; ++k)
            if (k < m) acc[k] += ((mk[k] >> code) & 1) ? -val : val;
        }
      }
      for (int k = 0; k < m; ++k) {
        const double s = sblock_sum(acc[k], red);
        if (threadIdx.x == 0) B.out[2 + k0 + k] = s;
      }
      __syncthreads();
      small_rot<R>(psi, dim, G, rl, (R)-1);
      small_rot<R>(lam, dim, G, rl, (R)-1);
      __syncthreads();
    }
  }
}

template <typename R>
cudaError_t launch_batch(const BatchItem *items, int n_items, int max_qubits, int any_grad, cudaStream_t st) {
  using C2 = typename SVec2<R>::type;
  if (n_items <= 0) return cudaSuccess;
  const size_t smem = sizeof(C2) * ((size_t)1 << max_qubits) * (any_grad ? 2 : 1);
  auto k = k_batch<R>;
  // per-function attribute shared by all host threads: the largest size any batch needs, set once
  // per device under a lock so that no launch on another thread overlaps a change of it
  const size_t smem_cap = sizeof(C2) * ((size_t)1 << SMALL_MAX_QUBITS) * 2;
  if (smem_cap > 48 * 1024) {
    static std::mutex mu;
    static std::set<int> done;
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    if (!done.count(d)) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap);
      if (e != cudaSuccess) return e;
      done.insert(d);
    }
  }
  int per_sm = 1, dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
  const int cap = sms * per_sm;
  const int grid = n_items < cap ? n_items : cap;
  k<<<grid, NT, smem, st>>>(items, n_items);
  return cudaGetLastError();
}

template cudaError_t launch_batch<float>(const BatchItem *, int, int, int, cudaStream_t);
template cudaError_t launch_batch<double>(const BatchItem *, int, int, int, cudaStream_t);

}  // namespace q2
