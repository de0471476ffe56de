// Batched-einsum IR of the engine (host side).
//
// A batched einsum is the quintuple (b, n, I_out, (I_in,j)_j, ((A^{i,j})_j)_i)
// of Sec. "Batched Einstein Summation"; every argument A is an idealized
// argument of a functional batched einsum (Def. "Functional Batched
// Einstein Summation"): either the identity lambda over a declared buffer
// or a lambda given by a producer expression over buffers, lambda
// parameters, literals and runtime scalars.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace be {

enum Status {
  OK = 0, EPARSE = 1, EINVALID = 2, ESHAPE = 3, EDTYPE = 4, ETOOMANY = 5,
  ENOTFOUND = 6, EDB = 7, EBUDGET = 8, ETIMEOUT = 9, ECUDA = 10,
  EUNSUPPORTED = 11, EARG = 12,
};

// DtypeRank of the induced-graph appendix; bfloat16 (absent there) is 9.
enum Dtype { I8 = 1, I32 = 2, I64 = 3, F16 = 4, F32 = 5, F64 = 6, C64 = 7, C128 = 8, BF16 = 9 };

const char *dtype_name(int dt);       // "float64", ...
int dtype_from_text(const std::string &s);  // 0 if unknown
int dtype_size(int dt);
int dtype_promote_rank(int dt);      // order used for result types

// producer expression node (postfix-friendly tree, children by index)
enum XOp : int8_t {
  X_NUM, X_SCALAR, X_PARAM, X_REF, X_NEG, X_ADD, X_SUB, X_MUL, X_DIV,
  X_SIN, X_COS, X_EXP, X_ABS, X_EQ, X_NE, X_SELECT,
};

struct XNode {
  XOp op;
  double num = 0.0;          // X_NUM
  int id = -1;               // X_SCALAR: scalar id; X_PARAM: param position; X_REF: buffer id
  std::vector<int> sub;      // X_REF: per buffer dim, >=0 param position, <0 -> constant -(sub+1)
  std::vector<int> kids;
};

struct Buffer {
  std::string name;
  int dtype = F64;
  std::vector<int64_t> shape;
};

struct Arg {
  std::string name;
  int dtype = F64;
  std::vector<int64_t> shape;   // the domain dom(A)
  int buffer = -1;              // identity lambda over this buffer, or -1
  std::vector<std::string> params;
  std::vector<XNode> nodes;     // functional body; nodes[root]
  int root = -1;
  bool functional() const { return buffer < 0; }
};

struct Einsum {
  std::string text;
  int b = 0, n = 0;
  std::vector<int8_t> out;                    // index letters 0..25
  std::vector<std::vector<int8_t>> in;        // per operand position
  std::vector<std::vector<int>> rows;         // b x n argument ids
  std::vector<Arg> args;                      // distinct idealized args, first appearance
  std::vector<Buffer> buffers;                // declared buffers, declaration order
  std::vector<std::string> scalars;           // runtime scalar names
  int64_t len[26] = {0};
  bool used[26] = {false};
  int out_dtype = F64;

  int n_index() const {
    int k = 0;
    for (bool u : used) k += u;
    return k;
  }
  std::vector<int64_t> out_shape() const {
    std::vector<int64_t> s;
    for (int8_t c : out) s.push_back(len[c]);
    return s;
  }
};

// Parse the textual spec; on error returns a status and fills err.
int parse(const std::string &text, Einsum &e, std::string &err);

// Soundness rules of Sec. "Preliminaries" for every row; fills e.len / used.
int check_sound(Einsum &e, std::string &err);

}  // namespace be
