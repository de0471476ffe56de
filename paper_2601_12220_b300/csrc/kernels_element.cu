// Element strategy (FP64 SIMT): batched einsums of the form
//
//     R_k[e, i] = sum_{r, j} D[r, i, j] * g_k[e, r] * u_k[e, j]
//
// with a small operator D shared by every row and per-element operands
// g_k, u_k streamed over a long element axis e -- the FEM action
// 'ij,ej->ei' (no r, no g) and the DG local gradient split by derivative
// direction (Sec. "Batched einsums in DG-FEM Operators", gradient tuple;
// Appendix C gradient pattern).  Following the transformation the paper
// describes for these kernels (loop hoisting to cut flops), the inner sum
// t[r, i] = sum_j D[r, i, j] u[e, j] is formed once per distinct u and
// reused by every row that shares it, then contracted with g_k.
//
// Layout: a persistent grid; each CTA stages D once in shared memory and
// then walks element tiles.  Per tile the u producers are evaluated while
// loading (e.g. u = sin(a) * b, fused into the operand load) into shared
// memory together with g; threads then own (e, i) output points, so the
// stores of R_k[e, i] are contiguous.
#include "exec.hpp"

namespace be {

namespace {

__device__ __forceinline__ double prod_value(const EProd &q, int64_t e, int k) {
  double a = q.a.ptr[e * q.a.se + k * q.a.sk];
  if (q.kind == 0) return a;
  double b = q.b.ptr[e * q.b.se + k * q.b.sk];
  if (q.kind == 2) return a * b;
  return sin(a) * b;
}

__global__ void __launch_bounds__(256) element_kernel(const __grid_constant__ EParams p) {
  extern __shared__ double smem[];
  const int R = p.R, NI = p.NI, NJ = p.NJ, TE = p.tile_e;
  double *Ds = smem;                                   // [R][NI][NJ]
  double *Us = Ds + R * NI * NJ;                       // [groups][TE][NJ]
  double *Gs = Us + p.n_groups * TE * NJ;              // [rows][TE][R]
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int idx = tid; idx < R * NI * NJ; idx += nt) {
    int r = idx / (NI * NJ), rem = idx % (NI * NJ);
    int i = rem / NJ, j = rem % NJ;
    Ds[idx] = p.D[r * p.sr + i * p.si + j * p.sj];
  }

  const int64_t n_tiles = (p.E + TE - 1) / TE;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t e0 = tile * TE;
    const int te = (int)((p.E - e0) < TE ? (p.E - e0) : TE);
    __syncthreads();   // D ready / previous tile consumed
    for (int idx = tid; idx < p.n_groups * te * NJ; idx += nt) {
      int g = idx / (te * NJ), rem = idx % (te * NJ);
      int el = rem / NJ, j = rem % NJ;
      Us[(g * TE + el) * NJ + j] = prod_value(p.groups[g], e0 + el, j);
    }
    if (p.has_g) {
      for (int idx = tid; idx < p.n_rows * te * R; idx += nt) {
        int k = idx / (te * R), rem = idx % (te * R);
        int el = rem / R, r = rem % R;
        const EView &v = p.rows[k].g;
        Gs[(k * TE + el) * R + r] = v.ptr[(e0 + el) * v.se + r * v.sk];
      }
    }
    __syncthreads();
    for (int item = tid; item < te * NI; item += nt) {
      const int el = item / NI, i = item % NI;
      for (int g = 0; g < p.n_groups; ++g) {
        double t[EM_MAXR];
        const double *u = Us + (g * TE + el) * NJ;
        for (int r = 0; r < R; ++r) {
          const double *d = Ds + (r * NI + i) * NJ;
          double acc = 0.0;
          for (int j = 0; j < NJ; ++j) acc = fma(d[j], u[j], acc);
          t[r] = acc;
        }
        for (int k = 0; k < p.n_rows; ++k) {
          if (p.rows[k].group != g) continue;
          double acc;
          if (p.has_g) {
            const double *gg = Gs + (k * TE + el) * R;
            acc = 0.0;
            for (int r = 0; r < R; ++r) acc = fma(gg[r], t[r], acc);
          } else {
            acc = t[0];
          }
          p.rows[k].out[(e0 + el) * NI + i] = acc;
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_element(const EParams &p, int grid, int block, cudaStream_t s) {
  size_t smem = sizeof(double) * ((size_t)p.R * p.NI * p.NJ + (size_t)p.n_groups * p.tile_e * p.NJ +
                                  (size_t)p.n_rows * p.tile_e * p.R);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  static bool attr = false;
  if (!attr) {
    cudaError_t st = cudaFuncSetAttribute(element_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (st != cudaSuccess) return st;
    attr = true;
  }
  element_kernel<<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace be
