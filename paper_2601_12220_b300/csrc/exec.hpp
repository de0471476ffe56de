// Execution layer: operand views, producer programs, kernel parameter
// blocks and the launchers of every strategy.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "ir.hpp"

namespace be {

// ---------------------------------------------------------------- generic

#define GMAXL 16      // distinct index letters an executed einsum may use
#define GMAXOPS 8     // operands per einsum on the generic path
#define GMAXINS 48    // producer instructions per einsum (all operands)
#define GSTACK 8      // producer evaluation stack depth

// One producer instruction.  X_REF reads ptr + sum_L coef[L] * value(L)
// (as dtype); X_PARAM pushes value(letter); X_SCALAR pushes scalars[letter].
struct GIns {
  int32_t op, dtype, letter, pad;
  double num;
  const char *ptr;
  int64_t coef[GMAXL];
};

struct GOp {
  int32_t kind;      // 0: strided view (ptr, coef, dtype); 1: producer program
  int32_t dtype;
  int32_t prog_begin, prog_len;
  const char *ptr;
  int64_t coef[GMAXL];
};

// Tiled form of a two-operand row (mode 3): C[b, m, n] = sum_k A[b, m, k] B[b, k, n]
// over a GEMM view of the letters -- M: output letters only A's offset
// depends on, N: output letters only B's offset depends on, batch: output
// letters both depend on, K: every contracted letter.  Each list runs
// outermost first; a CTA computes a tile x tile block of one batch value.
// Every output sums its terms in increasing k, whatever the tile, so the
// launcher may pick the side: large tiles reuse staged operands more, small
// ones give more CTAs (FP64, whose pipe is the bound, wants many).
#define GT_MAX 64
#define GT_K 16

struct GGemm {
  int32_t nm, nn, nk, nb;           // letters per role
  int32_t m[GMAXL], n[GMAXL], k[GMAXL], b[GMAXL];
  int64_t M, N, K, B;               // extents
  int64_t tiles_m, tiles_n, tiles;  // tiles per batch value along M, N; all tiles
  int64_t out_coef[GMAXL];          // dense output offset per letter
  int32_t a_kmajor, b_kmajor;       // consecutive threads load along K (else along M / N)
  int32_t tile;                     // 32 or 64 outputs per side
  int32_t pad;
};

// tile side (16, 32 or 64; 64 for FP32 only) and the tile counts it gives
inline void set_gemm_tile(GGemm &g, int tile) {
  g.tile = tile;
  g.tiles_m = (g.M + tile - 1) / tile;
  g.tiles_n = (g.N + tile - 1) / tile;
  g.tiles = g.B * g.tiles_m * g.tiles_n;
}

struct alignas(16) GParams {
  int32_t n_ops, n_letters, n_out, n_con;
  int64_t len[GMAXL];
  int32_t out_letter[GMAXL];
  int32_t con_letter[GMAXL];
  int64_t total_out, total_con;
  void *out;
  int32_t out_dtype;
  int32_t mode;         // 0 thread, 1 warp, 2 CTA per output (by contraction length), 3 GEMM tiles
  int32_t fast;         // 1: <= 4 operands, all views of the output's dtype, <= 4 contracted letters
  int32_t n_hoist;      // fast rows: the last n_hoist operands do not depend on a contracted letter
  int32_t n_inv;        // fast rows, modes 0-2: the n_inv operands before those do not depend on
                        // the innermost contracted letter
  int32_t pad_inv;
  GGemm gemm;           // mode 3 only
  double scalars[8];
  GOp ops[GMAXOPS];
  GIns ins[GMAXINS];
};

cudaError_t launch_generic(const GParams &p, cudaStream_t s);

// ---------------------------------------------------------------- persistent

// one unit of work of the persistent executor: outputs [start, start+count) of row
// a tile of outputs of one row; dep[q] >= 0 names a row whose every tile
// (need[q] of them) must be finished before this tile starts (a factored
// step reading an intermediate)
struct PTile {
  int32_t row, pad;
  int64_t start, count;
  int32_t dep[2], need[2];
};

// done[row] counts the finished tiles of each row (zeroed before a launch
// whose tiles have dependencies; may be null when none has); status
// receives BE_ETIMEOUT if a dependency wait gives up after wait_limit SM
// cycles (0: about one second)
cudaError_t launch_persistent(const GParams *rows, const PTile *tiles, int64_t n_tiles, unsigned long long *counter,
                              unsigned int *done, int *status, long long wait_limit, int grid, int block,
                              cudaStream_t s);

// ---------------------------------------------------------------- element

#define EM_MAXROWS 16
#define EM_MAXN 64
#define EM_MAXR 4
#define EM_MAXK 128     // flat contracted extent S * NJ0 of the stacked form
#define EM_MAXX 4       // terms x of a stacked producer

// strided 2-index view x[e, k] = ptr[e * se + k * sk]
struct EView {
  const double *ptr;
  int64_t se, sk;
};

// strided view over (e, s, j): ptr[e * se + s * ss + j * sj]
struct ESView {
  const double *ptr;
  int64_t se, ss, sj;
};

// producer of a per-element operand: 0 view a; 1 sin(a) * b; 2 a * b;
// 3 (stacked) v[e, s, j] = sum_{x < X} A_x[e, s, j] * B_x[e, s, j], read at
// the flat index k = s * NJ0 + j (EParams::NJ0)
struct EProd {
  int32_t kind, X;
  EView a, b;
  ESView A[EM_MAXX], B[EM_MAXX];
};

struct ERow {
  EView g;          // g[e, r] (unused without r)
  int32_t group;    // index of this row's u-producer group
  int32_t pad;
  double *out;      // dense out[e, i]
};

// R_k[e, i] = sum_{r, j} D[r, i, j] g_k[e, r] u_k[e, j] with D[r, i, j] at
// D[r * sr + i * si + j * sj].  In the stacked form (NJ0 > 0: R = 1, no g)
// the contracted index is the flat k = s * NJ0 + j < NJ over two letters
// of D, read at D[i * si + s * sr + j * sj].
struct EParams {
  const double *D;
  int64_t sr, si, sj;          // D[r, i, j] strides
  int32_t R, NI, NJ, has_g;
  int64_t E;
  int32_t n_rows, n_groups, tile_e, NJ0;
  ERow rows[EM_MAXROWS];
  EProd groups[EM_MAXROWS];
};

// whether a producer group evaluates sin(a) * b (the kernels fill their
// sine tables only then)
__host__ __device__ inline bool uses_sin(const EParams &p) {
  for (int g = 0; g < p.n_groups; ++g)
    if (p.groups[g].kind == 1) return true;
  return false;
}

// shared-memory doubles (or float pairs) of the FP64 and double-float
// element kernels: the operator, one producer group's operand tile (groups
// are staged one after another) and every row's geometric factors
__host__ __device__ inline size_t element_smem_words(const EParams &p) {
  // D, the produced operand of one tile, g per row, and in the stacked form
  // the tile's A_x[e, s] when they do not depend on j (converted once)
  const size_t stacked = p.NJ0 > 0 ? (size_t)p.tile_e * EM_MAXX * (p.NJ / p.NJ0) : 0;
  return (size_t)p.R * p.NI * p.NJ + (size_t)p.tile_e * p.NJ + (size_t)p.n_rows * p.tile_e * p.R + stacked;
}
// budget for those words: 200 KB less the double-float kernel's sine table
#define EM_SMEM_BUDGET (190 * 1024)

// offset of D[r, i, k] (flat k in the stacked form)
__host__ __device__ inline int64_t d_offset(const EParams &p, int r, int i, int k) {
  if (p.NJ0 > 0) {
    const int s = k / p.NJ0;
    return (int64_t)i * p.si + (int64_t)s * p.sr + (int64_t)(k - s * p.NJ0) * p.sj;
  }
  return (int64_t)r * p.sr + (int64_t)i * p.si + (int64_t)k * p.sj;
}

cudaError_t launch_element(const EParams &p, int grid, int block, cudaStream_t s);
// same strategy in double-float arithmetic on the FP32 pipe (FP64 accuracy)
cudaError_t launch_element_df(const EParams &p, int grid, int block, cudaStream_t s);
// the double-float variant for small operators (NI, NJ <= 8, not stacked):
// one thread per element; fp64_share16 / 16 of the elements run on the FP64
// pipe beside the double-float ones
// default FP64 share of the small-operator kernel, in sixteenths (measured on
// the FEM action at E = 2^24)
#define SMALL_FP64_SHARE16 8
bool element_df_small(const EParams &p);
cudaError_t launch_element_df_small(const EParams &p, int fp64_share16, cudaStream_t s);
int element_df_block(const EParams &p);   // block size matching one tile's work items
// same strategy with t = u D^T as a digit-split GEMM on the tcgen05 tensor
// cores (every output certified within 1e-12 S, the rest recomputed in
// FP64); status receives BE_ETIMEOUT if a bounded wait expires, wait_limit
// is in SM cycles (0: about one second)
bool element_tc_supported(const EParams &p, std::string &why);
cudaError_t launch_element_tc(const EParams &p, int *status, long long wait_limit, cudaStream_t s);

}  // namespace be
