// Generic strategy: one thread per output element of one einsum, any
// notation.  Evaluates Eq. (1) directly -- the output indices come from the
// thread's element, the contracted indices run as an odometer -- and each
// operand value is either a strided load or the result of the operand's
// producer program (the lambda of a functional batched einsum, evaluated at
// the access, i.e. fused into the load).  Accumulates in the output's type.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "exec.hpp"

namespace be {

namespace {

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

template <typename T>
__global__ void __launch_bounds__(256) generic_kernel(const __grid_constant__ GParams p) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < p.total_out; o += stride) {
    int64_t val[GMAXL];
    for (int L = 0; L < GMAXL; ++L) val[L] = 0;
    int64_t rem = o;
    for (int d = p.n_out - 1; d >= 0; --d) {
      int L = p.out_letter[d];
      val[L] = rem % p.len[L];
      rem /= p.len[L];
    }
    T acc = (T)0;
    for (int64_t it = 0; it < p.total_con; ++it) {
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
      acc += prod;
      for (int t = p.n_con - 1; t >= 0; --t) {
        int L = p.con_letter[t];
        if (++val[L] < p.len[L]) break;
        val[L] = 0;
      }
    }
    if (p.out_dtype == F64) ((double *)p.out)[o] = (double)acc;
    else ((float *)p.out)[o] = (float)acc;
  }
}

}  // namespace

cudaError_t launch_generic(const GParams &p, cudaStream_t s) {
  if (p.total_out == 0) return cudaSuccess;
  int block = 256;
  int64_t blocks = (p.total_out + block - 1) / block;
  int grid = (int)(blocks < 148 * 16 ? blocks : 148 * 16);
  if (p.out_dtype == F64) generic_kernel<double><<<grid, block, 0, s>>>(p);
  else generic_kernel<float><<<grid, block, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace be
