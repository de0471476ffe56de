// Per-output-element evaluation of one einsum row (Eq. (1)): decode the
// output indices, run the contracted indices as an odometer, multiply the
// operand values (strided loads or producer programs evaluated at the
// access) and accumulate in the output's type.  Long contractions are split
// over a warp or a CTA with a fixed assignment and a fixed reduction order,
// so the result is deterministic.  Shared by the generic
// kernel and the persistent multi-instance executor, so both produce the
// same bits for the same row.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "exec.hpp"

namespace be {
namespace gen {

template <typename T>
__device__ __forceinline__ T load_as(const char *p, int dtype) {
  switch (dtype) {
    case F64: return (T)*(const double *)p;
    case F32: return (T)*(const float *)p;
    case F16: return (T)__half2float(*(const __half *)p);
    case BF16: return (T)__bfloat162float(*(const __nv_bfloat16 *)p);
    case I32: return (T)*(const int32_t *)p;
    case I64: return (T)*(const int64_t *)p;
    case I8: return (T)*(const int8_t *)p;
  }
  return (T)0;
}

__device__ __forceinline__ int esize(int dtype) {
  switch (dtype) {
    case I8: return 1;
    case F16: case BF16: return 2;
    case F32: case I32: return 4;
  }
  return 8;
}

template <typename T>
__device__ T eval_prog(const GParams &p, int begin, int count, const int64_t *val) {
  T st[GSTACK];
  int sp = 0;
  for (int k = begin; k < begin + count; ++k) {
    const GIns &in = p.ins[k];
    switch (in.op) {
      case X_NUM: st[sp++] = (T)in.num; break;
      case X_SCALAR: st[sp++] = (T)p.scalars[in.letter]; break;
      case X_PARAM: st[sp++] = (T)val[in.letter]; break;
      case X_REF: {
        int64_t off = 0;
        for (int L = 0; L < p.n_letters; ++L) off += in.coef[L] * val[L];
        st[sp++] = load_as<T>(in.ptr + off * esize(in.dtype), in.dtype);
        break;
      }
      case X_NEG: st[sp - 1] = -st[sp - 1]; break;
      case X_ADD: st[sp - 2] = st[sp - 2] + st[sp - 1]; --sp; break;
      case X_SUB: st[sp - 2] = st[sp - 2] - st[sp - 1]; --sp; break;
      case X_MUL: st[sp - 2] = st[sp - 2] * st[sp - 1]; --sp; break;
      case X_DIV: st[sp - 2] = st[sp - 2] / st[sp - 1]; --sp; break;
      case X_SIN: st[sp - 1] = sin(st[sp - 1]); break;
      case X_COS: st[sp - 1] = cos(st[sp - 1]); break;
      case X_EXP: st[sp - 1] = exp(st[sp - 1]); break;
      case X_ABS: st[sp - 1] = fabs(st[sp - 1]); break;
      case X_EQ: st[sp - 2] = (T)(st[sp - 2] == st[sp - 1]); --sp; break;
      case X_NE: st[sp - 2] = (T)(st[sp - 2] != st[sp - 1]); --sp; break;
      case X_SELECT: st[sp - 3] = st[sp - 3] != (T)0 ? st[sp - 2] : st[sp - 1]; sp -= 2; break;
    }
  }
  return st[0];
}

// contracted letters of val[] set to the digits of iteration index it
__device__ __forceinline__ void set_con(const GParams &p, int64_t *val, int64_t it) {
  for (int t = p.n_con - 1; t >= 0; --t) {
    const int L = p.con_letter[t];
    val[L] = it % p.len[L];
    it /= p.len[L];
  }
}

// advance the contracted odometer by s iterations (mixed-radix add)
__device__ __forceinline__ void add_con(const GParams &p, int64_t *val, int64_t s) {
  for (int t = p.n_con - 1; t >= 0 && s > 0; --t) {
    const int L = p.con_letter[t];
    int64_t v = val[L] + s;
    if (v < p.len[L]) {
      val[L] = v;
      return;
    }
    s = v / p.len[L];
    val[L] = v - s * p.len[L];
  }
}

template <typename T>
__device__ __forceinline__ T term(const GParams &p, const int64_t *val) {
  T prod = (T)1;
  for (int k = 0; k < p.n_ops; ++k) {
    const GOp &op = p.ops[k];
    T v;
    if (op.kind == 0) {
      int64_t off = 0;
      for (int L = 0; L < p.n_letters; ++L) off += op.coef[L] * val[L];
      v = load_as<T>(op.ptr + off * esize(op.dtype), op.dtype);
    } else {
      v = eval_prog<T>(p, op.prog_begin, op.prog_len, val);
    }
    prod *= v;
  }
  return prod;
}

// sum of the terms of output o over iterations first, first + stride, ...
template <typename T>
__device__ T contract(const GParams &p, int64_t o, int64_t first, int64_t stride) {
  int64_t val[GMAXL];
  for (int L = 0; L < GMAXL; ++L) val[L] = 0;
  int64_t rem = o;
  for (int d = p.n_out - 1; d >= 0; --d) {
    const int L = p.out_letter[d];
    val[L] = rem % p.len[L];
    rem /= p.len[L];
  }
  T acc = (T)0;
  if (first >= p.total_con) return acc;
  set_con(p, val, first);
  for (int64_t it = first; it < p.total_con; it += stride) {
    acc += term<T>(p, val);
    if (stride == 1) {
      for (int t = p.n_con - 1; t >= 0; --t) {
        const int L = p.con_letter[t];
        if (++val[L] < p.len[L]) break;
        val[L] = 0;
      }
    } else {
      add_con(p, val, stride);
    }
  }
  return acc;
}

// Sum of the terms of output o over the contiguous iterations [lo, hi) for a
// row whose operands are all plain views of type T (GParams::fast), with
// NV operands that move along the innermost contracted letter followed by NI
// that do not (GParams::n_inv): within a run the NV operands' products are
// summed and the run's sum is multiplied once by the NI operands' product.  The output letters give each operand's base; the
// iterations then run as runs of the innermost contracted letter: a run is
// a tight loop of typed loads at a 32-bit stride and one multiply-add per
// term, and the outer letters advance (an odometer) between runs, adding a
// letter's coefficient on each step and taking len * coefficient off when
// it wraps.  GParams::fast guarantees that the contraction count and every
// in-operand offset fit in 32 bits.  Iterations run in the same order as
// contract() with stride 1.
template <typename T, int NV, int NI>
__device__ T contract_runs(const GParams &p, const int64_t *base, int lo, int hi) {
  constexpr int NOPS = NV + NI;
  const T *q[NOPS];
#pragma unroll
  for (int k = 0; k < NOPS; ++k) q[k] = (const T *)p.ops[k].ptr + base[k];
  // innermost contracted letter: digit din of lin, stride s[k]; outer
  // letters cl[t]: digit dig[t] of ln[t]
  int din = 0, lin = 1, s[NOPS];
  int dig[3] = {0, 0, 0}, ln[3] = {1, 1, 1}, cl[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < NOPS; ++k) s[k] = 0;
  int it = lo;
  if (p.n_con > 0) {
    const int L = p.con_letter[p.n_con - 1];
    lin = (int)p.len[L];
    din = it % lin;
    it /= lin;
#pragma unroll
    for (int k = 0; k < NOPS; ++k) {
      s[k] = (int)p.ops[k].coef[L];
      q[k] += (int64_t)s[k] * din;
    }
  }
#pragma unroll
  for (int t = 2; t >= 0; --t) {
    if (t < p.n_con - 1) {
      cl[t] = p.con_letter[t];
      ln[t] = (int)p.len[cl[t]];
      dig[t] = it % ln[t];
      it /= ln[t];
#pragma unroll
      for (int k = 0; k < NOPS; ++k) q[k] += p.ops[k].coef[cl[t]] * dig[t];
    }
  }
  T acc = (T)0;
  int i = lo;
  while (i < hi) {
    const int n = min(lin - din, hi - i);
    if constexpr (NI == 0) {
#pragma unroll 4
      for (int c = 0; c < n; ++c) {
        T prod = q[0][c * s[0]];
#pragma unroll
        for (int k = 1; k < NV; ++k) prod *= q[k][c * s[k]];
        acc += prod;
      }
    } else {
      T run = (T)0;
#pragma unroll 4
      for (int c = 0; c < n; ++c) {
        T prod = q[0][c * s[0]];
#pragma unroll
        for (int k = 1; k < NV; ++k) prod *= q[k][c * s[k]];
        run += prod;
      }
      T inv = q[NV][0];
#pragma unroll
      for (int k = NV + 1; k < NOPS; ++k) inv *= q[k][0];
      acc += inv * run;
    }
    i += n;
    if (i >= hi) break;
    // the innermost letter wrapped (the run started at digit din): back to
    // its digit 0, carry outward
#pragma unroll
    for (int k = 0; k < NOPS; ++k) q[k] -= (int64_t)s[k] * din;
    din = 0;
#pragma unroll
    for (int t = 2; t >= 0; --t) {
      if (t >= p.n_con - 1) continue;
      ++dig[t];
#pragma unroll
      for (int k = 0; k < NOPS; ++k) q[k] += p.ops[k].coef[cl[t]];
      if (dig[t] < ln[t]) break;
      dig[t] = 0;
#pragma unroll
      for (int k = 0; k < NOPS; ++k) q[k] -= p.ops[k].coef[cl[t]] * ln[t];
    }
  }
  return acc;
}

// Offsets of output o's element in each operand of a fast row (output
// letters only), with 32-bit divisions when the output count fits.
__device__ __forceinline__ void out_offsets(const GParams &p, int64_t o, int64_t off[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) off[k] = 0;
  if (p.total_out < ((int64_t)1 << 31)) {
    uint32_t rem = (uint32_t)o;
    for (int d = p.n_out - 1; d >= 0; --d) {
      const int L = p.out_letter[d];
      const uint32_t n = (uint32_t)p.len[L], t = rem / n, v = rem - t * n;
      rem = t;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < p.n_ops) off[k] += p.ops[k].coef[L] * (int64_t)v;
    }
  } else {
    int64_t rem = o;
    for (int d = p.n_out - 1; d >= 0; --d) {
      const int L = p.out_letter[d];
      const int64_t t = rem / p.len[L], v = rem - t * p.len[L];
      rem = t;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < p.n_ops) off[k] += p.ops[k].coef[L] * v;
    }
  }
}

// The sum over [lo, hi) of the operands that move with the contraction,
// times the hoisted operands (GParams::n_hoist, constant over the sum).
template <typename T>
__device__ __forceinline__ T contract_fast(const GParams &p, int64_t o, int64_t lo, int64_t hi) {
  if (lo >= hi) return (T)0;
  int64_t base[4];
  out_offsets(p, o, base);
  T acc;
  const int l = (int)lo, h = (int)hi;
  switch ((p.n_ops - p.n_hoist) * 4 + p.n_inv) {   // (run operands, of them constant within a run)
    case 4: acc = contract_runs<T, 1, 0>(p, base, l, h); break;
    case 8: acc = contract_runs<T, 2, 0>(p, base, l, h); break;
    case 9: acc = contract_runs<T, 1, 1>(p, base, l, h); break;
    case 12: acc = contract_runs<T, 3, 0>(p, base, l, h); break;
    case 13: acc = contract_runs<T, 2, 1>(p, base, l, h); break;
    case 14: acc = contract_runs<T, 1, 2>(p, base, l, h); break;
    case 17: acc = contract_runs<T, 3, 1>(p, base, l, h); break;
    case 18: acc = contract_runs<T, 2, 2>(p, base, l, h); break;
    case 19: acc = contract_runs<T, 1, 3>(p, base, l, h); break;
    default: acc = contract_runs<T, 4, 0>(p, base, l, h); break;
  }
#pragma unroll
  for (int k = 1; k < 4; ++k)
    if (k >= p.n_ops - p.n_hoist && k < p.n_ops) acc *= ((const T *)p.ops[k].ptr)[base[k]];
  return acc;
}

// iterations [lo, hi) of lane v of nv (32 or 256): contiguous chunks
__device__ __forceinline__ void chunk_of(int64_t total, int v, int nv, int64_t &lo, int64_t &hi) {
  const int64_t c = nv == 32 ? (total + 31) >> 5 : (total + 255) >> 8;
  lo = min(total, (int64_t)v * c);
  hi = min(total, lo + c);
}

// One output, evaluated the same way by every kernel that uses the row:
//   mode 0: one thread, iterations in order;
//   mode 1: one warp, lane l takes iterations l, l+32, ..., then a fixed
//           butterfly sum (lane 0's value is used);
//   mode 2: one CTA, virtual lane v in [0, 256) takes v, v+256, ..., then a
//           fixed tree over the 256 partials in shared memory.
// Modes 1 and 2 must be called by the whole warp / CTA; the result is valid
// in lane 0 / thread 0.
// (rows with GParams::fast give each lane or virtual lane a contiguous
// chunk of the iterations instead of every 32nd / 256th one; the chunks are
// fixed, so the result is still deterministic)
template <typename T>
__device__ __forceinline__ T out_thread(const GParams &p, int64_t o) {
  return p.fast ? contract_fast<T>(p, o, 0, p.total_con) : contract<T>(p, o, 0, 1);
}

template <typename T>
__device__ __forceinline__ T out_warp(const GParams &p, int64_t o) {
  const int lane = threadIdx.x & 31;
  T v;
  if (p.fast) {
    int64_t lo, hi;
    chunk_of(p.total_con, lane, 32, lo, hi);
    v = contract_fast<T>(p, o, lo, hi);
  } else {
    v = contract<T>(p, o, lane, 32);
  }
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <typename T>
__device__ __forceinline__ T out_block(const GParams &p, int64_t o, double *red) {
  for (int v = threadIdx.x; v < 256; v += blockDim.x) {
    if (p.fast) {
      int64_t lo, hi;
      chunk_of(p.total_con, v, 256, lo, hi);
      red[v] = (double)contract_fast<T>(p, o, lo, hi);
    } else {
      red[v] = (double)contract<T>(p, o, v, 256);
    }
  }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    for (int v = threadIdx.x; v < w; v += blockDim.x) red[v] = (double)((T)red[v] + (T)red[v + w]);
    __syncthreads();
  }
  T r = (T)red[0];
  __syncthreads();
  return r;
}

// Mode 3: one TM x TM tile of the GEMM view (GGemm) of a row with two
// operands in its sum (a hoisted third operand multiplies each finished sum).
// Per K-slice of 16, the CTA stages A[m, k] and B[k, n] in shared memory
// (loaded along the role in which the operand is contiguous), with the
// offsets of the slice's m, n and k values computed once from the letters'
// digits; each of the 16 x 16 threads then accumulates an R x R block of
// outputs (R = TM / 16), every output summing its terms in increasing k (so
// the result does not depend on which kernel runs the tile).  Must be called
// by the whole CTA.
// one mixed-radix digit of x (v = x mod len, x = x / len), in 32-bit
// arithmetic when both fit; the outermost digit needs no division (x is
// below its length)
__device__ __forceinline__ void digit_step(int64_t &x, int64_t len, int64_t &v) {
  if ((uint64_t)x < 0x80000000ull && (uint64_t)len < 0x80000000ull) {
    const uint32_t xu = (uint32_t)x, lu = (uint32_t)len, q = xu / lu;
    v = (int64_t)(xu - q * lu);
    x = (int64_t)q;
  } else {
    v = x % len;
    x /= len;
  }
}

constexpr int GEMM_SMEM = 2 * GT_K * (GT_MAX + 2) * 8 + (6 * GT_MAX + 2 * GT_K) * 8;

template <typename T, int TM>
__device__ void gemm_tile(const GParams &p, int64_t tile, unsigned char *sm) {
  constexpr int R = TM / 16;                        // outputs per thread along each side
  constexpr int S = TM + 16 / (int)sizeof(T);       // padded row of a staged slice
  constexpr int PER = TM * GT_K / 256;              // staged values per thread and operand
  const GGemm &g = p.gemm;
  // uniform over the CTA: a tile outside the grid, or a CTA of other than
  // 256 threads (the staging below assigns its tables to fixed thread
  // ranges; the host never launches such a CTA for GEMM rows)
  if (tile >= g.tiles || blockDim.x != 256) return;
  T *As = (T *)sm;                                  // [GT_K][S]
  T *Bs = As + GT_K * S;                            // [GT_K][S]
  int64_t *offAm = (int64_t *)(sm + 2 * GT_K * (GT_MAX + 2) * 8);
  int64_t *offCm = offAm + GT_MAX, *offBn = offCm + GT_MAX, *offCn = offBn + GT_MAX;
  int64_t *offAk = offCn + GT_MAX, *offBk = offAk + GT_K;
  int64_t *offHm = offBk + GT_K, *offHn = offHm + GT_MAX;   // the hoisted operand, if any
  const int tid = threadIdx.x;
  const int64_t *ca = p.ops[0].coef, *cb = p.ops[1].coef;
  const bool hoist = p.n_hoist > 0;
  const int64_t *ch = p.ops[hoist ? 2 : 0].coef;
  int64_t r = tile;
  const int64_t nt = r % g.tiles_n;
  r /= g.tiles_n;
  const int64_t mt = r % g.tiles_m;
  r /= g.tiles_m;
  int64_t baseA = 0, baseB = 0, baseC = 0, baseH = 0;
  for (int d = g.nb - 1; d >= 0; --d) {
    const int L = g.b[d];
    const int64_t v = r % p.len[L];
    r /= p.len[L];
    baseA += ca[L] * v;
    baseB += cb[L] * v;
    baseC += g.out_coef[L] * v;
    baseH += ch[L] * v;
  }
  const int64_t m0 = mt * TM, n0 = nt * TM;
  const int vm = (int)min((int64_t)TM, g.M - m0), vn = (int)min((int64_t)TM, g.N - n0);
  if (tid < TM) {
    int64_t x = m0 + tid, oa = 0, oc = 0, oh = 0;
    if (tid < vm)
      for (int d = g.nm - 1; d >= 0; --d) {
        const int L = g.m[d];
        int64_t v = x;
        if (d > 0) digit_step(x, p.len[L], v);
        oa += ca[L] * v;
        oc += g.out_coef[L] * v;
        oh += ch[L] * v;
      }
    offAm[tid] = oa;
    offCm[tid] = oc;
    offHm[tid] = oh;
  } else if (tid >= 64 && tid < 64 + TM) {
    const int t = tid - 64;
    int64_t x = n0 + t, ob = 0, oc = 0, oh = 0;
    if (t < vn)
      for (int d = g.nn - 1; d >= 0; --d) {
        const int L = g.n[d];
        int64_t v = x;
        if (d > 0) digit_step(x, p.len[L], v);
        ob += cb[L] * v;
        oc += g.out_coef[L] * v;
        oh += ch[L] * v;
      }
    offBn[t] = ob;
    offCn[t] = oc;
    offHn[t] = oh;
  }
  const T *A = (const T *)p.ops[0].ptr + baseA, *B = (const T *)p.ops[1].ptr + baseB;
  const int tm = tid >> 4, tn = tid & 15;
  // threads whose whole block lies outside the tile skip the arithmetic
  const bool active = tm * R < vm && tn * R < vn;
  T acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = (T)0;
  for (int64_t k0 = 0; k0 < g.K; k0 += GT_K) {
    const int vk = (int)min((int64_t)GT_K, g.K - k0);
    __syncthreads();   // the previous slice is consumed; the m / n tables are written
    if (tid >= 128 && tid < 128 + GT_K) {
      const int t = tid - 128;
      int64_t x = k0 + t, oa = 0, ob = 0;
      if (t < vk)
        for (int d = g.nk - 1; d >= 0; --d) {
          const int L = g.k[d];
          int64_t v = x;
          if (d > 0) digit_step(x, p.len[L], v);
          oa += ca[L] * v;
          ob += cb[L] * v;
        }
      offAk[t] = oa;
      offBk[t] = ob;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q;
      const int kk = g.a_kmajor ? e % GT_K : e / TM, mm = g.a_kmajor ? e / GT_K : e % TM;
      As[kk * S + mm] = (kk < vk && mm < vm) ? A[offAm[mm] + offAk[kk]] : (T)0;
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q;
      const int kk = g.b_kmajor ? e % GT_K : e / TM, nn = g.b_kmajor ? e / GT_K : e % TM;
      Bs[kk * S + nn] = (kk < vk && nn < vn) ? B[offBn[nn] + offBk[kk]] : (T)0;
    }
    __syncthreads();
    if (!active) continue;
    for (int kk = 0; kk < vk; ++kk) {
      T a[R], b[R];
      if constexpr (sizeof(T) * R >= 16) {          // 16-byte loads (the rows are 16-byte aligned)
#pragma unroll
        for (int i = 0; i < R; i += 16 / (int)sizeof(T)) {
          const float4 av = *(const float4 *)&As[kk * S + tm * R + i], bv = *(const float4 *)&Bs[kk * S + tn * R + i];
          memcpy(a + i, &av, 16);
          memcpy(b + i, &bv, 16);
        }
      } else {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          a[i] = As[kk * S + tm * R + i];
          b[i] = Bs[kk * S + tn * R + i];
        }
      }
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] += a[i] * b[j];
    }
  }
  T *C = (T *)p.out + baseC;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int m = tm * R + i;
    if (m >= vm) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int n = tn * R + j;
      if (n >= vn) continue;
      // the hoisted operand multiplies the finished sum
      C[offCm[m] + offCn[n]] = hoist ? acc[i][j] * ((const T *)p.ops[2].ptr)[baseH + offHm[m] + offHn[n]] : acc[i][j];
    }
  }
  __syncthreads();   // the tables and slices are free for the next tile
}

// every output of [start, start + count) of row p, by the row's mode (GEMM
// tiles [start, start + count) in mode 3)
__device__ __forceinline__ void eval_range(const GParams &p, int64_t start, int64_t count, double *red,
                                           unsigned char *gsm) {
  const int64_t end = start + count;
  if (p.mode == 3) {   // [start, end) are GEMM tiles
    for (int64_t t = start; t < end; ++t) {
      if (p.out_dtype == F64) {
        if (p.gemm.tile == 16) gemm_tile<double, 16>(p, t, gsm);
        else gemm_tile<double, 32>(p, t, gsm);
      } else {
        if (p.gemm.tile == 16) gemm_tile<float, 16>(p, t, gsm);
        else if (p.gemm.tile == 32) gemm_tile<float, 32>(p, t, gsm);
        else gemm_tile<float, 64>(p, t, gsm);
      }
    }
  } else if (p.mode == 0) {
    for (int64_t o = start + threadIdx.x; o < end; o += blockDim.x) {
      if (p.out_dtype == F64) ((double *)p.out)[o] = out_thread<double>(p, o);
      else ((float *)p.out)[o] = out_thread<float>(p, o);
    }
  } else if (p.mode == 1) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int64_t o = start + warp; o < end; o += nw) {
      if (p.out_dtype == F64) {
        double v = out_warp<double>(p, o);
        if (lane == 0) ((double *)p.out)[o] = v;
      } else {
        float v = out_warp<float>(p, o);
        if (lane == 0) ((float *)p.out)[o] = v;
      }
    }
  } else {
    for (int64_t o = start; o < end; ++o) {
      if (p.out_dtype == F64) {
        double v = out_block<double>(p, o, red);
        if (threadIdx.x == 0) ((double *)p.out)[o] = v;
      } else {
        float v = out_block<float>(p, o, red);
        if (threadIdx.x == 0) ((float *)p.out)[o] = v;
      }
    }
  }
}

}  // namespace gen
}  // namespace be
