// RaiseToBatchedEinsum: a loop-nest kernel -> the text of the functional
// batched einsum it computes (be_parse grammar), with the loop name of every
// index letter and the output array of every row.
#pragma once

#include <string>
#include <vector>

#include "ir.hpp"

namespace be {

struct Raised {
  std::string spec;                       // be_parse text
  std::vector<std::string> loop_names;    // letter k ('a' + k) -> loop name
  std::vector<std::string> outputs;       // row -> output array
};

int raise_kernel(const std::string &text, Raised &r, std::string &err);

}  // namespace be
