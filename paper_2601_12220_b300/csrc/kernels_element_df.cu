// Element strategy on the FP32 pipe: the same batched einsums as
// element_kernel (R_k[e,i] = sum_{r,j} D[r,i,j] g_k[e,r] u_k[e,j], D shared,
// Sec. "Batched einsums in DG-FEM Operators", and the stacked form of the
// divergence and face mass), with the same hoisting
// t[r,i] = sum_j D[r,i,j] u[e,j] once per distinct u, but every operation in
// double-float (df) arithmetic: D, u and g are held as float pairs, the dot
// products accumulate exactly through TwoSum with the cross terms in a
// second float, and the fused producer u = sin(a) * b is evaluated with the
// df sine (full-circle table).  Results reach FP64 accuracy (about 2^-46 of the absolute
// contraction) while the FP64 pipe only adds the two halves of each output.
#include <algorithm>

#include "df_math.cuh"
#include "exec.hpp"
#include "launch_attr.hpp"
#include "launch_rec.hpp"

namespace be {

namespace {

using dfm::df;

// the producer's value at (e, k) in double-float.  The operands are loaded
// first and range-tested together; when all pass (the usual case) the
// conversions and the sine run without tests or out-of-line calls.
__device__ __forceinline__ df prod_df(const EProd &q, int64_t e, int k, int NJ0, const float2 *sin_tab) {
  if (q.kind == 3) {   // stacked: sum_x A_x[e, s, j] * B_x[e, s, j] at k = s * NJ0 + j, in df
    const int s = k / NJ0, j = k - s * NJ0;
    double av[EM_MAXX], bv[EM_MAXX];
    bool ok = true;
#pragma unroll
    for (int x = 0; x < EM_MAXX; ++x) {
      av[x] = x < q.X ? q.A[x].ptr[e * q.A[x].se + s * q.A[x].ss + j * q.A[x].sj] : 0.0;
      bv[x] = x < q.X ? q.B[x].ptr[e * q.B[x].se + s * q.B[x].ss + j * q.B[x].sj] : 0.0;
      ok = ok && dfm::df_fast_ok(av[x]) && dfm::df_fast_ok(bv[x]);
    }
    float sh = 0.f, sl = 0.f;
    if (ok) {
#pragma unroll
      for (int x = 0; x < EM_MAXX; ++x)
        if (x < q.X) dfm::dot_acc(sh, sl, dfm::df_from_double_fast(av[x]), dfm::df_from_double_fast(bv[x]));
    } else {
#pragma unroll
      for (int x = 0; x < EM_MAXX; ++x)
        if (x < q.X) dfm::dot_acc(sh, sl, dfm::df_from_double(av[x]), dfm::df_from_double(bv[x]));
    }
    return dfm::two_sum(sh, sl);
  }
  const double a = q.a.ptr[e * q.a.se + k * q.a.sk];
  if (q.kind == 0) return dfm::df_fast_ok(a) ? dfm::df_from_double_fast(a) : dfm::df_from_double(a);
  const double b = q.b.ptr[e * q.b.se + k * q.b.sk];
  if (q.kind == 2) {
    if (dfm::df_fast_ok(a) && dfm::df_fast_ok(b))
      return dfm::df_mul(dfm::df_from_double_fast(a), dfm::df_from_double_fast(b));
    return dfm::df_mul(dfm::df_from_double(a), dfm::df_from_double(b));
  }
  if (dfm::sin_fast_ok(a) && dfm::df_fast_ok(b))
    return dfm::df_mul(dfm::df_sin_tab2_fast(a, sin_tab), dfm::df_from_double_fast(b));
  return dfm::df_mul(dfm::df_sin_tab2(a, sin_tab), dfm::df_from_double(b));
}

// the producer's value at (e, k) in FP64 (the small-operator kernel's FP64
// share): a view, a * b, or sin(a) * b with the df sine rounded to FP64
__device__ __forceinline__ double prod_fp64(const EProd &q, int64_t e, int k, const float2 *sin_tab) {
  const double a = q.a.ptr[e * q.a.se + k * q.a.sk];
  if (q.kind == 0) return a;
  const double b = q.b.ptr[e * q.b.se + k * q.b.sk];
  if (q.kind == 2) return a * b;
  return dfm::df_to_double(dfm::sin_fast_ok(a) ? dfm::df_sin_tab2_fast(a, sin_tab) : dfm::df_sin_tab2(a, sin_tab)) * b;
}

constexpr int DF_EPT = 4;   // elements per thread in the contraction phase

__global__ void __launch_bounds__(512, 2) element_df_kernel(const __grid_constant__ EParams p) {
  extern __shared__ float2 smf[];
  const int R = p.R, NI = p.NI, NJ = p.NJ, TE = p.tile_e;
  float2 *Ds = smf;                                   // [R][NI][NJ]
  float2 *Us = Ds + R * NI * NJ;                      // [TE][NJ], one producer group at a time
  float2 *Gs = Us + TE * NJ;                          // [rows][TE][R]
  float2 *Ac = Gs + p.n_rows * TE * R;                // stacked form: [TE][EM_MAXX][S]
  const int n_f2 = (int)element_smem_words(p);
  float2 *sin_tab = smf + n_f2;                       // full-circle sine table
  const int tid = threadIdx.x, nt = blockDim.x;
  if (uses_sin(p)) dfm::sin2_table_fill(sin_tab);

  for (int idx = tid; idx < R * NI * NJ; idx += nt) {
    const int r = idx / (NI * NJ), rem = idx % (NI * NJ);
    const int i = rem / NJ, j = rem % NJ;
    const df d = dfm::df_from_double(p.D[d_offset(p, r, i, j)]);
    Ds[idx] = make_float2(d.hi, d.lo);
  }

  const int64_t n_tiles = (p.E + TE - 1) / TE;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t e0 = tile * TE;
    const int te = (int)((p.E - e0) < TE ? (p.E - e0) : TE);
    __syncthreads();
    if (p.has_g) {
      for (int idx = tid; idx < p.n_rows * te * R; idx += nt) {
        const int k = idx / (te * R), rem = idx % (te * R);
        const int el = rem / R, r = rem % R;
        const EView &v = p.rows[k].g;
        const df gv = dfm::df_from_double(v.ptr[(e0 + el) * v.se + r * v.sk]);
        Gs[(k * TE + el) * R + r] = make_float2(gv.hi, gv.lo);
      }
    }
    // each item: one dof i for DF_EPT consecutive elements, so D[r, i, :] is
    // read once from shared memory for all of them
    const int groups_e = (te + DF_EPT - 1) / DF_EPT;
    for (int g = 0; g < p.n_groups; ++g) {
      if (g > 0) __syncthreads();   // the previous group's operand consumed
      const EProd &q = p.groups[g];
      bool a_no_j = q.kind == 3, b_no_s = q.kind == 3;
      for (int x = 0; x < EM_MAXX; ++x)
        if (x < q.X) {
          a_no_j = a_no_j && q.A[x].sj == 0;
          b_no_s = b_no_s && q.B[x].ss == 0;
        }
      if (a_no_j) {
        // stacked form whose A_x[e, s] do not depend on j (the metric terms
        // of the divergence, the face Jacobians of the face mass): each is
        // converted once per tile; a thread then forms v[e, s, j] for every
        // s of one (e, j), converting B_x[e, j] once when it does not depend
        // on s.  The same df operations as prod_df, in the same order.
        const int NJ0 = p.NJ0, S = NJ / NJ0;
        for (int idx = tid; idx < te * q.X * S; idx += nt) {
          const int el = idx / (q.X * S), rem = idx % (q.X * S), x = rem / S, sx = rem % S;
          const double a = q.A[x].ptr[(e0 + el) * q.A[x].se + sx * q.A[x].ss];
          const df d = dfm::df_fast_ok(a) ? dfm::df_from_double_fast(a) : dfm::df_from_double(a);
          Ac[(el * EM_MAXX + x) * S + sx] = make_float2(d.hi, d.lo);
        }
        __syncthreads();
        for (int idx = tid; idx < te * NJ0; idx += nt) {
          const int el = idx / NJ0, j = idx % NJ0;
          const int64_t e = e0 + el;
          df bx[EM_MAXX];
#pragma unroll
          for (int x = 0; x < EM_MAXX; ++x) {
            bx[x] = df{0.f, 0.f};
            if (b_no_s && x < q.X) {
              const double b = q.B[x].ptr[e * q.B[x].se + j * q.B[x].sj];
              bx[x] = dfm::df_fast_ok(b) ? dfm::df_from_double_fast(b) : dfm::df_from_double(b);
            }
          }
          for (int sx = 0; sx < S; ++sx) {
            float sh = 0.f, sl = 0.f;
#pragma unroll
            for (int x = 0; x < EM_MAXX; ++x) {
              if (x >= q.X) continue;
              df b = bx[x];
              if (!b_no_s) {
                const double bv = q.B[x].ptr[e * q.B[x].se + sx * q.B[x].ss + j * q.B[x].sj];
                b = dfm::df_fast_ok(bv) ? dfm::df_from_double_fast(bv) : dfm::df_from_double(bv);
              }
              const float2 a = Ac[(el * EM_MAXX + x) * S + sx];
              dfm::dot_acc(sh, sl, df{a.x, a.y}, b);
            }
            const df v = dfm::two_sum(sh, sl);
            Us[el * NJ + sx * NJ0 + j] = make_float2(v.hi, v.lo);
          }
        }
      } else {
        for (int idx = tid; idx < te * NJ; idx += nt) {
          const int el = idx / NJ, j = idx % NJ;
          const df u = prod_df(q, e0 + el, j, p.NJ0, sin_tab);
          Us[el * NJ + j] = make_float2(u.hi, u.lo);
        }
      }
      __syncthreads();
      for (int item = tid; item < groups_e * NI; item += nt) {
        const int eg = item / NI, i = item % NI;
        const int el0 = eg * DF_EPT;
        const int nq = min(DF_EPT, te - el0);
        df t[DF_EPT][EM_MAXR];
        const float2 *u0 = Us + el0 * NJ;
#pragma unroll
        for (int r = 0; r < EM_MAXR; ++r) {
          if (r >= R) break;
          const float2 *d = Ds + (r * NI + i) * NJ;
          float s[DF_EPT], c[DF_EPT];
#pragma unroll
          for (int q = 0; q < DF_EPT; ++q) s[q] = c[q] = 0.f;
          for (int j = 0; j < NJ; ++j) {
            const float2 dj = d[j];
#pragma unroll
            for (int q = 0; q < DF_EPT; ++q) {
              const float2 uq = u0[q * NJ + j];       // beyond te: unused values, never stored
              dfm::dot_acc(s[q], c[q], df{dj.x, dj.y}, df{uq.x, uq.y});
            }
          }
#pragma unroll
          for (int q = 0; q < DF_EPT; ++q) t[q][r] = dfm::fast_two_sum(s[q], c[q]);
        }
        for (int k = 0; k < p.n_rows; ++k) {
          if (p.rows[k].group != g) continue;
#pragma unroll
          for (int q = 0; q < DF_EPT; ++q) {
            if (q >= nq) break;
            const int el = el0 + q;
            df acc;
            if (p.has_g) {
              const float2 *gg = Gs + (k * TE + el) * R;
              float s = 0.f, c = 0.f;
#pragma unroll
              for (int r = 0; r < EM_MAXR; ++r)
                if (r < R) dfm::dot_acc(s, c, df{gg[r].x, gg[r].y}, t[q][r]);
              acc = dfm::fast_two_sum(s, c);
            } else {
              acc = t[q][0];
            }
            p.rows[k].out[(e0 + el) * NI + i] = dfm::df_to_double(acc);
          }
        }
      }
    }
  }
}

// Small operators (NI, NJ <= NB, R <= RM <= 4; e.g. the FEM action's 4 x 4
// D): one thread per (producer group: blockIdx.y, element) keeps u[e, :] and
// t[r, i] in registers, so the streamed operands are read and the outputs
// written once, coalesced across the warp, with no tile staging.  B300's
// FP64 pipe and its FP32 pipe work side by side: the first blocks64 blocks
// of each group evaluate the elements [0, E64) as FP64 multiply-add chains,
// the others the elements [E64, E) in double-float; block dispatch
// interleaves the two kinds on every SM.  In the double-float part, entries
// beyond NI / NJ are zero, which adds nothing to a compensated sum, so every
// output is the same sequence of df operations as in element_df_kernel.
template <int NB, int RM>
__global__ void __launch_bounds__(256, (NB == 4 && RM == 1) ? 4 : 2)
    element_df_small_kernel(const __grid_constant__ EParams p, int64_t E64, int blocks64) {
  __shared__ float2 Ds[RM * NB * NB];   // [r][i][j] as df
  __shared__ double Dd[RM * NB * NB];   // the same in FP64
  __shared__ float2 sin_tab[dfm::SIN2_N];
  const int R = p.R, NI = p.NI, NJ = p.NJ;
  if (uses_sin(p)) dfm::sin2_table_fill(sin_tab);
  for (int idx = threadIdx.x; idx < RM * NB * NB; idx += blockDim.x) {
    const int r = idx / (NB * NB), i = (idx / NB) % NB, j = idx % NB;
    const double v = (r < R && i < NI && j < NJ) ? p.D[d_offset(p, r, i, j)] : 0.0;
    const df d = dfm::df_from_double(v);
    Ds[idx] = make_float2(d.hi, d.lo);
    Dd[idx] = v;
  }
  __syncthreads();
  const int g = blockIdx.y;                     // producer group
  const EProd &q = p.groups[g];
  const bool fp64 = (int)blockIdx.x < blocks64;
  const int64_t lo = fp64 ? 0 : E64, hi = fp64 ? E64 : p.E;
  const int64_t b0 = fp64 ? blockIdx.x : blockIdx.x - blocks64;
  const int64_t nb = fp64 ? blocks64 : (int64_t)gridDim.x - blocks64;
  for (int64_t e = lo + b0 * blockDim.x + threadIdx.x; e < hi; e += nb * blockDim.x) {
    if (fp64) {
      double u[NB], t[RM][NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) u[j] = j < NJ ? prod_fp64(q, e, j, sin_tab) : 0.0;
#pragma unroll
      for (int r = 0; r < RM; ++r) {
        if (r >= R) break;
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < NB; ++j)
            if (j < NJ) acc = fma(Dd[(r * NB + i) * NB + j], u[j], acc);
          t[r][i] = acc;
        }
      }
      for (int k = 0; k < p.n_rows; ++k) {
        if (p.rows[k].group != g) continue;
        const EView &v = p.rows[k].g;
        double *out = p.rows[k].out + e * NI;
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          if (i >= NI) break;
          double acc = t[0][i];
          if (p.has_g) {
            acc = 0.0;
#pragma unroll
            for (int r = 0; r < RM; ++r)
              if (r < R) acc = fma(v.ptr[e * v.se + r * v.sk], t[r][i], acc);
          }
          out[i] = acc;
        }
      }
      continue;
    }
    df u[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) u[j] = j < NJ ? prod_df(q, e, j, 0, sin_tab) : df{0.f, 0.f};
    df t[RM][NB];
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      if (r >= R) break;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        float sh = 0.f, sl = 0.f;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          const float2 d = Ds[(r * NB + i) * NB + j];
          dfm::dot_acc(sh, sl, df{d.x, d.y}, u[j]);
        }
        t[r][i] = dfm::fast_two_sum(sh, sl);
      }
    }
    for (int k = 0; k < p.n_rows; ++k) {
      if (p.rows[k].group != g) continue;
      df gk[RM];
      if (p.has_g) {
        const EView &v = p.rows[k].g;
#pragma unroll
        for (int r = 0; r < RM; ++r)
          if (r < R) gk[r] = dfm::df_from_double(v.ptr[e * v.se + r * v.sk]);
      }
      double *out = p.rows[k].out + e * NI;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (i >= NI) break;
        df acc = t[0][i];
        if (p.has_g) {
          float sh = 0.f, sl = 0.f;
#pragma unroll
          for (int r = 0; r < RM; ++r)
            if (r < R) dfm::dot_acc(sh, sl, gk[r], t[r][i]);
          acc = dfm::fast_two_sum(sh, sl);
        }
        out[i] = dfm::df_to_double(acc);
      }
    }
  }
}

}  // namespace

bool element_df_small(const EParams &p) { return p.NJ0 == 0 && p.R <= EM_MAXR && p.NI <= 8 && p.NJ <= 8; }

cudaError_t launch_element_df_small(const EParams &p, int fp64_share16, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // x: elements (grid-stride; the first b64 blocks take the FP64 share,
  // fp64_share16 / 16 of the elements), y: producer groups
  fp64_share16 = std::max(0, std::min(16, fp64_share16));
  const int64_t per_group = std::max<int64_t>(2, (int64_t)sms * 8 / std::max(1, p.n_groups) + 1);
  const int64_t E64 = std::min(p.E, (p.E * fp64_share16 / 16 + 255) / 256 * 256);
  const int64_t need64 = (E64 + 255) / 256, needdf = (p.E - E64 + 255) / 256;
  const int64_t b64 = E64 > 0 ? std::max<int64_t>(1, std::min<int64_t>(need64, per_group * fp64_share16 / 16)) : 0;
  const int64_t bdf = E64 < p.E ? std::max<int64_t>(1, std::min<int64_t>(needdf, per_group - b64)) : 0;
  const dim3 grid((unsigned)std::max<int64_t>(1, b64 + bdf), (unsigned)p.n_groups);
  const bool r1 = p.R == 1;
  if (p.NI <= 4 && p.NJ <= 4) {
    return r1 ? be_launch(element_df_small_kernel<4, 1>, grid, dim3(256), 0, s, p, E64, (int)b64)
              : be_launch(element_df_small_kernel<4, EM_MAXR>, grid, dim3(256), 0, s, p, E64, (int)b64);
  } else {
    return r1 ? be_launch(element_df_small_kernel<8, 1>, grid, dim3(256), 0, s, p, E64, (int)b64)
              : be_launch(element_df_small_kernel<8, EM_MAXR>, grid, dim3(256), 0, s, p, E64, (int)b64);
  }
}

int element_df_block(const EParams &p) {
  const int items = (p.tile_e + DF_EPT - 1) / DF_EPT * p.NI;
  return std::min(512, std::max(32, (items + 31) / 32 * 32));
}

cudaError_t launch_element_df(const EParams &p, int grid, int block, cudaStream_t s) {
  if (p.tile_e % DF_EPT) return cudaErrorInvalidValue;          // element groups never straddle a tile
  const size_t smem = sizeof(float2) * (element_smem_words(p) + dfm::SIN2_N);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  static std::atomic<uint64_t> attr{0};
  cudaError_t st = smem_limit_once((const void *)element_df_kernel, 200 * 1024, attr);
  if (st != cudaSuccess) return st;
  return be_launch(element_df_kernel, dim3(grid), dim3(block), smem, s, p);
}

}  // namespace be
