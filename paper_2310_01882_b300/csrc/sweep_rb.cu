// sweep_rb.cu -- compiled configurations of the red-black Gauss-Seidel
// kernel (RbCfg, sweep_rb_kernel.cuh): T = 2 colour stages (one red-black
// sweep) per pass for every policy, T = 4 (two sweeps) for FP32 and BF16
// storage.  RbCfg<policy, T, R, WY, S, CTAs per SM>; the first entry of each
// list (the default) is the fastest measured on a 512^3 grid.
#include "sweep_launch.cuh"

namespace stencil {

int sweep_variants_rb(int policy, int T, const SweepVariant** out) {
  static const SweepVariant res2[] = {
      variant<PolResident, RbCfg<PolResident, 2, 4, 4, 4, 2>>(),
      variant<PolResident, RbCfg<PolResident, 2, 4, 4, 5, 2>>(),
      variant<PolResident, RbCfg<PolResident, 2, 4, 8, 5, 1>>(),
      variant<PolResident, RbCfg<PolResident, 2, 2, 8, 4, 2>>(),
      variant<PolResident, RbCfg<PolResident, 2, 2, 8, 6, 1>>(),
      variant<PolResident, RbCfg<PolResident, 2, 8, 4, 4, 1>>(),
      variant<PolResident, RbCfg<PolResident, 2, 2, 6, 4, 3>>(),
  };
  static const SweepVariant fix2[] = {
      variant<PolFixed, RbCfg<PolFixed, 2, 4, 4, 4, 2>>(),
      variant<PolFixed, RbCfg<PolFixed, 2, 4, 8, 5, 1>>(),
  };
  static const SweepVariant f642[] = {
      variant<PolF64, RbCfg<PolF64, 2, 2, 8, 6, 1>>(),
  };
  static const SweepVariant f322[] = {
      variant<PolF32, RbCfg<PolF32, 2, 4, 4, 5, 4>>(),
      variant<PolF32, RbCfg<PolF32, 2, 4, 4, 4, 4>>(),
      variant<PolF32, RbCfg<PolF32, 2, 4, 4, 6, 3>>(),
      variant<PolF32, RbCfg<PolF32, 2, 8, 4, 4, 2>>(),
      variant<PolF32, RbCfg<PolF32, 2, 8, 8, 4, 1>>(),
      variant<PolF32, RbCfg<PolF32, 2, 4, 8, 4, 2>>(),
      variant<PolF32, RbCfg<PolF32, 2, 4, 8, 6, 1>>(),
  };
  static const SweepVariant f324[] = {
      variant<PolF32, RbCfg<PolF32, 4, 4, 4, 6, 2>>(),
      variant<PolF32, RbCfg<PolF32, 4, 4, 8, 6, 1>>(),
      variant<PolF32, RbCfg<PolF32, 4, 2, 8, 6, 2>>(),
      variant<PolF32, RbCfg<PolF32, 4, 2, 4, 7, 1>>(),
  };
  static const SweepVariant b162[] = {
      variant<PolBF16, RbCfg<PolBF16, 2, 4, 4, 4, 4>>(),
      variant<PolBF16, RbCfg<PolBF16, 2, 4, 4, 5, 4>>(),
      variant<PolBF16, RbCfg<PolBF16, 2, 4, 4, 6, 3>>(),
      variant<PolBF16, RbCfg<PolBF16, 2, 8, 4, 4, 2>>(),
      variant<PolBF16, RbCfg<PolBF16, 2, 8, 8, 4, 1>>(),
      variant<PolBF16, RbCfg<PolBF16, 2, 4, 8, 4, 2>>(),
      variant<PolBF16, RbCfg<PolBF16, 2, 4, 8, 6, 1>>(),
  };
  static const SweepVariant b164[] = {
      variant<PolBF16, RbCfg<PolBF16, 4, 4, 4, 6, 2>>(),
      variant<PolBF16, RbCfg<PolBF16, 4, 4, 8, 6, 1>>(),
      variant<PolBF16, RbCfg<PolBF16, 4, 2, 8, 6, 2>>(),
      variant<PolBF16, RbCfg<PolBF16, 4, 2, 4, 7, 1>>(),
  };
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
