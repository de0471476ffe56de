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
// then walks element tiles.  Per tile g is staged for every row, then each
// distinct u producer in turn is evaluated while loading (e.g. u = sin(a) *
// b, fused into the operand load) into shared memory and contracted;
// threads own (e, i) output points, so the stores of R_k[e, i] are
// contiguous.
#include "exec.hpp"
#include "launch_attr.hpp"
#include "launch_rec.hpp"

namespace be {

namespace {

__device__ __forceinline__ double prod_value(const EProd &q, int64_t e, int k, int NJ0) {
  if (q.kind == 3) {   // stacked: sum_x A_x[e, s, j] * B_x[e, s, j] at k = s * NJ0 + j
    const int s = k / NJ0, j = k - s * NJ0;
    double acc = 0.0;
    for (int x = 0; x < q.X; ++x)
      acc = fma(q.A[x].ptr[e * q.A[x].se + s * q.A[x].ss + j * q.A[x].sj],
                q.B[x].ptr[e * q.B[x].se + s * q.B[x].ss + j * q.B[x].sj], acc);
    return acc;
  }
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
  double *Us = Ds + R * NI * NJ;                       // [TE][NJ], one producer group at a time
  double *Gs = Us + TE * NJ;                           // [rows][TE][R]
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int idx = tid; idx < R * NI * NJ; idx += nt) {
    int r = idx / (NI * NJ), rem = idx % (NI * NJ);
    int i = rem / NJ, j = rem % NJ;
    Ds[idx] = p.D[d_offset(p, r, i, j)];
  }

  const int64_t n_tiles = (p.E + TE - 1) / TE;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t e0 = tile * TE;
    const int te = (int)((p.E - e0) < TE ? (p.E - e0) : TE);
    __syncthreads();   // D ready / previous tile consumed
    if (p.has_g) {
      for (int idx = tid; idx < p.n_rows * te * R; idx += nt) {
        int k = idx / (te * R), rem = idx % (te * R);
        int el = rem / R, r = rem % R;
        const EView &v = p.rows[k].g;
        Gs[(k * TE + el) * R + r] = v.ptr[(e0 + el) * v.se + r * v.sk];
      }
    }
    for (int g = 0; g < p.n_groups; ++g) {
      if (g > 0) __syncthreads();   // the previous group's operand consumed
      for (int idx = tid; idx < te * NJ; idx += nt) {
        int el = idx / NJ, j = idx % NJ;
        Us[el * NJ + j] = prod_value(p.groups[g], e0 + el, j, p.NJ0);
      }
      __syncthreads();
      for (int item = tid; item < te * NI; item += nt) {
        const int el = item / NI, i = item % NI;
        double t[EM_MAXR];
        const double *u = Us + el * NJ;
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
  size_t smem = sizeof(double) * element_smem_words(p);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  static std::atomic<uint64_t> attr{0};
  cudaError_t st = smem_limit_once((const void *)element_kernel, 200 * 1024, attr);
  if (st != cudaSuccess) return st;
  return be_launch(element_kernel, dim3(grid), dim3(block), smem, s, p);
}

}  // namespace be
