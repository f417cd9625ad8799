// Host-side problem setup of libsos (no device code).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sos.h"
#include "sos_plan.h"

namespace sos {

// Everything the device needs, in host memory, for a batch of instances.
struct HostPlan {
  int32_t n_inst = 0;
  int64_t NX = 0, M = 0;
  int32_t TL = 0;
  int64_t n_linv = 0;
  std::vector<InstInfo> inst;
  std::vector<BlockDesc> blocks;
  // rows (size M)
  std::vector<double> b, pinv, h2;
  std::vector<int32_t> row_inst;
  std::vector<int32_t> row_ptr;   // M + 1, plain Gram entries per row
  std::vector<uint32_t> row_ent;  // entry index | kOffDiagBit
  // entries (size NX): row of a plain Gram entry, -1 otherwise
  std::vector<int32_t> ent_row;
  // low-rank part A_L: CSC (TL + 1) and CSR (M + 1)
  std::vector<int32_t> lr_ptr, lr_row;
  std::vector<double> lr_val;
  std::vector<int32_t> lrr_ptr, lrr_col;
  std::vector<double> lrr_val;
  std::vector<int64_t> lr_ent;    // x index of each low-rank column
  std::vector<int32_t> lr_inst;
  std::vector<double> lr_c;       // c on the column (w_i for free variables, 0 else)
  std::vector<double> lr_g;       // A_L^T h_2 (Sherman-Morrison data)
  std::vector<double> linv;       // per-instance L^{-1}
  std::vector<int64_t> x_inst_start;  // NX boundaries (n_inst + 1)
};

// Builds the plan; returns SOS_OK or an SOS_ERR_* code with a message.
// weighted_form: 0 choose per program by eq. (42), 1 weighted blocks directly,
// 2 extra polynomials (end of Section II).
int build_plan(const sos_program* progs, int32_t n_progs, HostPlan& plan, std::string& err, int weighted_form = 0);

// Message returned by sos_last_error(NULL) (shared by every entry point
// that has no handle).
void set_global_error(const std::string& msg);

// Graded monomials of eq. (4); returns the count.
int64_t enumerate_monomials(int32_t n_vars, int32_t degree, int32_t* out, int64_t capacity);

}  // namespace sos
