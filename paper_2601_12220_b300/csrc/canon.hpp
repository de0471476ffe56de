// Canonicalization of batched einsums (Alg. 1) and the induced graph of
// Appendix B.
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "ir.hpp"

namespace be {

// Node colours of the induced-graph appendix (Eq. for c_i).
enum Color { C_ARG = 1, C_INDEX = 2, C_ACC_IN = 3, C_ACC_OUT = 4, C_OUTPUT = 5,
             C_ARGPOS = 6, C_DTYPE = 7, C_LENGTH = 8, C_DIM = 9 };

struct Graph {
  int n = 0;
  std::vector<int> color;                    // 1..9
  std::vector<std::pair<int, int>> edges;    // directed (from, to)
  std::vector<int> dtype_of;                 // iota_dtype: node -> DtypeRank (0 if not a dtype node)
  std::vector<int64_t> length_of;            // iota_length: node -> axis length (-1 otherwise)
  // bookkeeping of the numbering chosen by ToInducedGraph
  std::vector<int> arg_node, index_node;     // per arg id / per letter (-1 unused)
  std::vector<int> row_node, pos_node;       // outputs (rows) and operand positions
  std::vector<std::vector<std::vector<int>>> acc_in_node;  // [row][pos][dim]
  std::vector<int> acc_out_node;             // per output dim
};

// Appendix B.1: batched einsum -> induced graph (Eq. for N^IDG, the edge
// sets E_*, and the colouring).
Graph to_induced_graph(const Einsum &e);

// Compliance conditions of Appendix B.2.  Returns 0 if all hold, else the
// number k of the first failing condition (Ck).
int graph_check(const Graph &g);

// Appendix B.2 Steps 1-11: a compliant graph -> batched einsum whose index
// k is named by letter k and whose argument k is "A<k>".  iota_index and
// iota_arg of the reconstruction are returned (node -> 0-based order).
int to_batched_einsum(const Graph &g, Einsum &out, std::vector<int> &index_order,
                      std::vector<int> &arg_order, std::string &err);

struct Canon {
  Einsum form;                       // C(e): letters a.., args A0..
  std::string key;                   // printed normal form
  std::vector<int64_t> tokens;       // T(C(e))
  std::vector<int> sigma_index;      // canonical letter k -> user letter
  std::vector<int> sigma_arg;        // canonical arg k -> user arg id
  std::vector<std::string> sigma_arg_name;  // canonical arg k -> user arg name
  std::vector<int> sigma_row;        // canonical row q -> user row
  std::vector<int> sigma_pos;        // canonical position p -> user position
  std::vector<int> relabel;          // RelabelingMap on the induced graph of e
  int graph_nodes = 0;
};

// Alg. 1.  GetCanonLabel is realised by an exact lexicographic search
// (C_lex) over operand and row orders; see canon.cpp.
int canonicalize(const Einsum &e, Canon &c, std::string &err);

std::string key_text(const Einsum &f);

}  // namespace be
