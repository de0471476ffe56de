// Element strategy on the FP32 pipe: the same batched einsums as
// element_kernel (R_k[e,i] = sum_{r,j} D[r,i,j] g_k[e,r] u_k[e,j], D shared,
// Sec. "Batched einsums in DG-FEM Operators"), with the same hoisting
// t[r,i] = sum_j D[r,i,j] u[e,j] once per distinct u, but every operation in
// double-float (df) arithmetic: D, u and g are held as float pairs, the dot
// products accumulate exactly through TwoSum with the cross terms in a
// second float, and the fused producer u = sin(a) * b is evaluated with the
// df sine.  Results reach FP64 accuracy (about 2^-46 of the absolute
// contraction) while the FP64 pipe only adds the two halves of each output.
#include "df_math.cuh"
#include "exec.hpp"

namespace be {

namespace {

using dfm::df;

__device__ __forceinline__ df prod_df(const EProd &q, int64_t e, int k) {
  const double a = q.a.ptr[e * q.a.se + k * q.a.sk];
  if (q.kind == 0) return dfm::df_from_double(a);
  const double b = q.b.ptr[e * q.b.se + k * q.b.sk];
  if (q.kind == 2) return dfm::df_mul(dfm::df_from_double(a), dfm::df_from_double(b));
  return dfm::df_mul(dfm::df_sin(a), dfm::df_from_double(b));
}

__global__ void __launch_bounds__(256) element_df_kernel(const __grid_constant__ EParams p) {
  extern __shared__ float2 smf[];
  const int R = p.R, NI = p.NI, NJ = p.NJ, TE = p.tile_e;
  float2 *Ds = smf;                                   // [R][NI][NJ]
  float2 *Us = Ds + R * NI * NJ;                      // [groups][TE][NJ]
  float2 *Gs = Us + p.n_groups * TE * NJ;             // [rows][TE][R]
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int idx = tid; idx < R * NI * NJ; idx += nt) {
    const int r = idx / (NI * NJ), rem = idx % (NI * NJ);
    const int i = rem / NJ, j = rem % NJ;
    const df d = dfm::df_from_double(p.D[r * p.sr + i * p.si + j * p.sj]);
    Ds[idx] = make_float2(d.hi, d.lo);
  }

  const int64_t n_tiles = (p.E + TE - 1) / TE;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t e0 = tile * TE;
    const int te = (int)((p.E - e0) < TE ? (p.E - e0) : TE);
    __syncthreads();
    for (int idx = tid; idx < p.n_groups * te * NJ; idx += nt) {
      const int g = idx / (te * NJ), rem = idx % (te * NJ);
      const int el = rem / NJ, j = rem % NJ;
      const df u = prod_df(p.groups[g], e0 + el, j);
      Us[(g * TE + el) * NJ + j] = make_float2(u.hi, u.lo);
    }
    if (p.has_g) {
      for (int idx = tid; idx < p.n_rows * te * R; idx += nt) {
        const int k = idx / (te * R), rem = idx % (te * R);
        const int el = rem / R, r = rem % R;
        const EView &v = p.rows[k].g;
        const df gv = dfm::df_from_double(v.ptr[(e0 + el) * v.se + r * v.sk]);
        Gs[(k * TE + el) * R + r] = make_float2(gv.hi, gv.lo);
      }
    }
    __syncthreads();
    for (int item = tid; item < te * NI; item += nt) {
      const int el = item / NI, i = item % NI;
      for (int g = 0; g < p.n_groups; ++g) {
        df t[EM_MAXR];
        const float2 *u = Us + (g * TE + el) * NJ;
        for (int r = 0; r < R; ++r) {
          const float2 *d = Ds + (r * NI + i) * NJ;
          float s = 0.f, c = 0.f;
          for (int j = 0; j < NJ; ++j) {
            const float2 dj = d[j], uj = u[j];
            dfm::dot_acc(s, c, df{dj.x, dj.y}, df{uj.x, uj.y});
          }
          t[r] = dfm::fast_two_sum(s, c);
        }
        for (int k = 0; k < p.n_rows; ++k) {
          if (p.rows[k].group != g) continue;
          df acc;
          if (p.has_g) {
            const float2 *gg = Gs + (k * TE + el) * R;
            float s = 0.f, c = 0.f;
            for (int r = 0; r < R; ++r) dfm::dot_acc(s, c, df{gg[r].x, gg[r].y}, t[r]);
            acc = dfm::fast_two_sum(s, c);
          } else {
            acc = t[0];
          }
          p.rows[k].out[(e0 + el) * NI + i] = dfm::df_to_double(acc);
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_element_df(const EParams &p, int grid, int block, cudaStream_t s) {
  const size_t smem = sizeof(float2) * ((size_t)p.R * p.NI * p.NJ + (size_t)p.n_groups * p.tile_e * p.NJ +
                                        (size_t)p.n_rows * p.tile_e * p.R);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  static bool attr = false;
  if (!attr) {
    cudaError_t st = cudaFuncSetAttribute(element_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (st != cudaSuccess) return st;
    attr = true;
  }
  element_df_kernel<<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace be
