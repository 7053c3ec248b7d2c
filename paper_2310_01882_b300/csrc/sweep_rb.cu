// sweep_rb.cu -- compiled configurations of the sweep kernel for red-black
// Gauss-Seidel (TbCfg<..., RB = true>): T = 2 stages (one red-black sweep)
// per pass for every policy, T = 4 (two sweeps) for FP32 and BF16 storage.
// TbCfg<policy, T, R, WY, S, CTAs per SM, red-black>.
#include "sweep_launch.cuh"

namespace stencil {

int sweep_variants_rb(int policy, int T, const SweepVariant** out) {
  static const SweepVariant res2[] = {
      variant<PolResident, TbCfg<PolResident, 2, 2, 4, 6, 3, true>>(),
      variant<PolResident, TbCfg<PolResident, 2, 4, 4, 5, 2, true>>(),
  };
  static const SweepVariant fix2[] = {variant<PolFixed, TbCfg<PolFixed, 2, 4, 4, 5, 2, true>>()};
  static const SweepVariant f642[] = {variant<PolF64, TbCfg<PolF64, 2, 4, 4, 5, 2, true>>()};
  static const SweepVariant f322[] = {
      variant<PolF32, TbCfg<PolF32, 2, 4, 8, 6, 2, true>>(),
      variant<PolF32, TbCfg<PolF32, 2, 8, 4, 5, 1, true>>(),
  };
  static const SweepVariant f324[] = {variant<PolF32, TbCfg<PolF32, 4, 4, 4, 7, 1, true>>()};
  static const SweepVariant b162[] = {variant<PolBF16, TbCfg<PolBF16, 2, 4, 8, 6, 2, true>>()};
  static const SweepVariant b164[] = {variant<PolBF16, TbCfg<PolBF16, 4, 4, 4, 7, 1, true>>()};
#define RET(arr)             \
  {                          \
    *out = arr;              \
    return sizeof(arr) / sizeof(arr[0]); \
  }
  if (T == 2) {
    if (policy == kPolResident) RET(res2);
    if (policy == kPolFixed) RET(fix2);
    if (policy == kPolF64) RET(f642);
    if (policy == kPolF32) RET(f322);
    if (policy == kPolBF16) RET(b162);
  } else if (T == 4) {
    if (policy == kPolF32) RET(f324);
    if (policy == kPolBF16) RET(b164);
  }
#undef RET
  *out = nullptr;
  return 0;
}

}  // namespace stencil
