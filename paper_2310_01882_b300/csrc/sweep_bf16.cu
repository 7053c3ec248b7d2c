// sweep_bf16.cu -- compiled configurations of the sweep kernel for bfloat16
// storage with binary32 arithmetic.  TbCfg<policy, T, R, WY, S, CTAs per SM>;
// at one sweep per pass the first shapes read both x neighbours from the
// staged plane (XSMEM), the fastest at 512^3 first.
#include "sweep_launch.cuh"

namespace stencil {

int sweep_variants_bf16(int T, const SweepVariant** out) {
  static const SweepVariant t1[] = {
      variant<PolBF16, TbCfg<PolBF16, 1, 8, 16, 8, 1, true, true>>(),
      variant<PolBF16, TbCfg<PolBF16, 1, 8, 16, 6, 1, true, true>>(),
      variant<PolBF16, TbCfg<PolBF16, 1, 8, 8, 4, 2, true, true>>(),
      variant<PolBF16, TbCfg<PolBF16, 1, 8, 8, 4, 2>>(),
      variant<PolBF16, TbCfg<PolBF16, 1, 8, 4, 5, 3>>(),
      variant<PolBF16, TbCfg<PolBF16, 1, 4, 8, 6, 3>>(),
      variant<PolBF16, TbCfg<PolBF16, 1, 4, 4, 5, 6>>(),
  };

  static const SweepVariant t2[] = {
      variant<PolBF16, TbCfg<PolBF16, 2, 8, 4, 5, 1>>(),
      variant<PolBF16, TbCfg<PolBF16, 2, 4, 8, 6, 2>>(),
      variant<PolBF16, TbCfg<PolBF16, 2, 4, 4, 6, 3>>(),
      variant<PolBF16, TbCfg<PolBF16, 2, 8, 4, 5, 3>>(),
      variant<PolBF16, TbCfg<PolBF16, 2, 4, 4, 5, 4>>(),
      variant<PolBF16, TbCfg<PolBF16, 2, 2, 8, 6, 3>>(),
  };
  static const SweepVariant t4[] = {
      variant<PolBF16, TbCfg<PolBF16, 4, 4, 4, 7, 1>>(),
      variant<PolBF16, TbCfg<PolBF16, 4, 2, 4, 8, 2>>(),
  };
  switch (T) {
    case 1: *out = t1; return sizeof(t1) / sizeof(t1[0]);
    case 2: *out = t2; return sizeof(t2) / sizeof(t2[0]);
    case 4: *out = t4; return sizeof(t4) / sizeof(t4[0]);
    default: *out = nullptr; return 0;
  }
}

}  // namespace stencil
