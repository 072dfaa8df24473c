// Host-side fault injection into the apply-program validator (no GPU).
//
// Every apply program (the packed stages of Z or Zinv) is checked on the host
// before the library uses it: after a build, a relocation, a restriction to a
// shard and a checkpoint load.  This harness builds a small valid program in
// host memory only (no device buffer is allocated; the matrix buffer's size is
// all the validator reads), checks that it is accepted, then corrupts one field
// of one block descriptor at a time and checks that each corruption is refused
// with VIE_EINVAL.  It links libvie.so and calls the library's own validator.
// Prints "ok <cases>" and exits 0, or names the first case that was not caught.
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "internal.h"

using namespace vie;

static OpDesc block(int64_t mat_off, int16_t in_sp, int64_t in_off, int16_t out_sp, int64_t out_off, int32_t M,
                    int32_t K, int32_t ld, int32_t acc) {
  OpDesc o{};
  o.mat_off = mat_off;
  o.in_space = in_sp;
  o.in_off = in_off;
  o.out_space = out_sp;
  o.out_off = out_off;
  o.M = M;
  o.K = K;
  o.ld = ld;
  o.accumulate = acc;
  return o;
}

// n = 8 unknowns, 6 coefficients; stage 0: a 2 x 4 block X[0:4] -> C[0:2] and a 4 x 4 leaf
// block X[4:8] -> Y[4:8]; stage 1: an 8 x 2 block C[0:2] -> Y[0:8] added.  Complex FP32
// factors, 8 bytes per element, rows padded to an even element count.
static void make_program(Program& p) {
  p.n = 8;
  p.ncoef = 6;
  p.factor_dtype = VIE_C64;
  p.stages.resize(2);
  p.stages[0].host_ops = {block(0, SP_X, 0, SP_C, 0, 2, 4, 4, 0), block(8, SP_X, 4, SP_Y, 4, 4, 4, 4, 0)};
  p.stages[0].mats.bytes = 8 * (8 + 16);
  p.stages[1].host_ops = {block(0, SP_C, 0, SP_Y, 0, 8, 2, 2, 1)};
  p.stages[1].mats.bytes = 8 * 16;
  for (Stage& st : p.stages) st.nops = (int64_t)st.host_ops.size();
}

static bool refused(const Program& p, std::string& why) {
  try {
    program_check(p);
  } catch (const Error& e) {
    if (e.status != VIE_EINVAL) {
      why = "wrong status " + std::to_string(e.status);
      return false;
    }
    return true;
  }
  why = "accepted";
  return false;
}

int main() {
  {
    Program p;
    make_program(p);
    try {
      program_check(p);
    } catch (const Error& e) {
      std::printf("FAIL: the valid program was refused: %s\n", e.msg.c_str());
      return 1;
    }
  }
  struct Case {
    const char* name;
    int stage, op;
    std::function<void(OpDesc&, Program&)> corrupt;
  };
  const std::vector<Case> cases = {
      {"matrix beyond the stage buffer", 0, 1, [](OpDesc& o, Program&) { o.mat_off = 10; }},
      {"odd matrix offset (16-byte rows)", 0, 1, [](OpDesc& o, Program&) { o.mat_off = 7; }},
      {"negative matrix offset", 0, 0, [](OpDesc& o, Program&) { o.mat_off = -2; }},
      {"odd leading dimension", 1, 0, [](OpDesc& o, Program&) { o.ld = 3; }},
      {"leading dimension below K", 0, 0, [](OpDesc& o, Program&) { o.ld = 2; }},
      {"negative row count", 0, 0, [](OpDesc& o, Program&) { o.M = -1; }},
      {"negative column count", 0, 0, [](OpDesc& o, Program&) { o.K = -4; }},
      {"input slice past the unknowns", 0, 1, [](OpDesc& o, Program&) { o.in_off = 5; }},
      {"negative input offset", 0, 0, [](OpDesc& o, Program&) { o.in_off = -1; }},
      {"output slice past the coefficients", 0, 0, [](OpDesc& o, Program&) { o.out_off = 5; }},
      {"output slice past the unknowns", 1, 0, [](OpDesc& o, Program&) { o.out_off = 1; }},
      {"unknown input space", 0, 0, [](OpDesc& o, Program&) { o.in_space = 3; }},
      {"unknown output space", 1, 0, [](OpDesc& o, Program&) { o.out_space = -1; }},
      {"coefficient space shrunk under a block", 1, 0, [](OpDesc&, Program& p) { p.ncoef = 1; }},
      {"stage buffer shorter than its blocks", 1, 0, [](OpDesc&, Program& p) { p.stages[1].mats.bytes = 8 * 14; }},
  };
  int n = 0;
  for (const Case& c : cases) {
    Program p;
    make_program(p);
    c.corrupt(p.stages[c.stage].host_ops[c.op], p);
    std::string why;
    if (!refused(p, why)) {
      std::printf("FAIL: %s: %s\n", c.name, why.c_str());
      return 1;
    }
    ++n;
  }
  std::printf("ok %d\n", n);
  return 0;
}
