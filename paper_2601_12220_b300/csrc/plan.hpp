// Planner interface: caller buffers, operand views and strategy planners.
#pragma once

#include <array>
#include <string>
#include <vector>

#include "exec.hpp"
#include "ir.hpp"

namespace be {

// mirror of be_config (include/be.h)
struct be_config_t {
  int32_t strategy;
  int32_t tile[4];
  int32_t stages;
  uint32_t stage_mask;
  int32_t vec;
  int32_t split;
};

// a caller buffer (device pointer for execution)
struct BufIn {
  void *ptr;
  const int64_t *strides;
  int32_t ndim;
  int32_t dtype;
};

// strided view of an operand at one position: ptr + sum_c coef[c] * value(c)
struct View {
  const char *ptr;
  int dtype;
  int64_t coef[26];
};

// dense split strategy: per row C = A B after flattening (M, K) x (K, N)
struct DenseRow {
  int argA, argB;
  const double *A, *B;
  int64_t lda, ska, ldb, snb;
  double *C;
  // affine producers: the operands are alA * A + beA and alB * B + beB
  double alA = 1.0, beA = 0.0, alB = 1.0, beB = 0.0;
};
struct DensePlan {
  int64_t M = 0, N = 0, K = 0;
  std::vector<DenseRow> rows;
};

bool arg_view(const Einsum &e, int arg, int pos, const std::vector<BufIn> &bufs, View &v);
int check_buffers(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs,
                  std::string &err);
int plan_generic_row(const Einsum &e, int row, const std::vector<BufIn> &bufs, const BufIn &out,
                     const std::vector<double> &scalars, GParams &p, std::string &err);
int plan_element(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs,
                 const be_config_t &cfg, EParams &p, std::string &why);
// scalars: the call's runtime scalars for the affine producers' coefficients,
// or nullptr when only the form is checked
int plan_dense(const Einsum &e, const std::vector<BufIn> &bufs, const std::vector<BufIn> &outs, DensePlan &p,
               std::string &why, const std::vector<double> *scalars = nullptr);

// ---- factored evaluation (a row as a sequence of two-operand einsums)

// One operand of a pairwise step: a strided view (pointer, dtype, the index
// letter of each dimension and its stride in elements).
struct FOp {
  const void *ptr = nullptr;
  int dtype = F64;
  std::vector<int8_t> letters;
  std::vector<int64_t> strides;
};

// Pairwise order of a row's n operands: step s combines slots steps[s][0]
// and steps[s][1] (slots 0..n-1 are the operands, slot n + s the result of
// step s), or, when steps[s][1] < 0, sums the letters that only slot
// steps[s][0] uses, into a dense row-major intermediate over letters[s];
// the last step's letters are the output's.  Costs count multiply-adds of
// one row.
struct FactorOrder {
  std::vector<std::array<int, 2>> steps;
  std::vector<std::vector<int8_t>> letters;
  double direct = 0, factored = 0;
  int64_t inter_elems = 0;      // elements of one row's intermediates
};

// The order with the fewest multiply-adds over all orders of pairwise and
// unary steps (n <= 5); false unless e has 2 to 5 operands and the order
// cuts the loop nest's multiply-adds at least `min_gain` times.
bool factor_order(const Einsum &e, double min_gain, FactorOrder &fo);
// operand pos of row `row` as a view; false for a functional argument other
// than a single buffer reference
bool operand_fop(const Einsum &e, int row, int pos, const std::vector<BufIn> &bufs, FOp &f);
// one step as a generic row writing `out` (dense row-major over
// out_letters): x with y, or x alone when y is null; out_dtype is the
// einsum's
int plan_factor_step(const Einsum &e, const FOp &x, const FOp *y, const std::vector<int8_t> &out_letters, void *out,
                     GParams &p, std::string &err);
// The same pairwise step planned for the split-precision tensor cores (a
// GEMM C = A B after flattening: the output's letters from one operand,
// then from the other, the contracted letters flattenable in both views);
// EUNSUPPORTED with the reason otherwise.
int plan_factor_step_dense(const Einsum &e, const FOp &x, const FOp &y, const std::vector<int8_t> &out_letters,
                           void *out, DensePlan &dp, std::string &why);

}  // namespace be
