// sweep_f64.cu -- compiled configurations of the sweep kernel for binary64
// storage: fixed point resident for the call, fixed point per pass, and
// binary64 arithmetic.  TbCfg<policy, T, R, WY, S, CTAs per SM>.
#include "sweep_launch.cuh"

namespace stencil {

int sweep_variants_f64(int policy, int T, const SweepVariant** out) {
  static const SweepVariant res1[] = {
      variant<PolResident, TbCfg<PolResident, 1, 4, 16, 5, 1>>(),
      variant<PolResident, TbCfg<PolResident, 1, 2, 16, 6, 1>>(),
      variant<PolResident, TbCfg<PolResident, 1, 2, 16, 5, 1>>(),
      variant<PolResident, TbCfg<PolResident, 1, 2, 8, 5, 2>>(),
      variant<PolResident, TbCfg<PolResident, 1, 4, 8, 5, 2>>(),
      variant<PolResident, TbCfg<PolResident, 1, 8, 4, 4, 3>>(),
      variant<PolResident, TbCfg<PolResident, 1, 8, 4, 6, 2>>(),
      variant<PolResident, TbCfg<PolResident, 1, 8, 8, 4, 1>>(),
      variant<PolResident, TbCfg<PolResident, 1, 1, 16, 5, 2>>(),
      variant<PolResident, TbCfg<PolResident, 1, 4, 4, 6, 4>>(),
  };
  static const SweepVariant res2[] = {
      variant<PolResident, TbCfg<PolResident, 2, 2, 4, 6, 3>>(),
      // stage-1 edge reads (30-column tiles): faster than the 28-column form
      // of this shape, 0.710 against 0.724 ms per sweep at 512^3
      variant<PolResident, TbCfg<PolResident, 2, 4, 4, 5, 2, true>>(),
  };
  static const SweepVariant fix1[] = {variant<PolFixed, TbCfg<PolFixed, 1, 2, 16, 5, 1>>(),
                                      variant<PolFixed, TbCfg<PolFixed, 1, 8, 4, 4, 3>>()};
  static const SweepVariant f641[] = {variant<PolF64, TbCfg<PolF64, 1, 8, 4, 4, 3>>()};
  if (policy == kPolResident && T == 1) { *out = res1; return sizeof(res1) / sizeof(res1[0]); }
  if (policy == kPolResident && T == 2) { *out = res2; return sizeof(res2) / sizeof(res2[0]); }
  if (policy == kPolFixed && T == 1) { *out = fix1; return sizeof(fix1) / sizeof(fix1[0]); }
  if (policy == kPolF64 && T == 1) { *out = f641; return 1; }
  *out = nullptr;
  return 0;
}

// The fixed-point residual (PolResid) through the same kernel: one pass, the
// first configuration the default.
int sweep_variants_resid(const SweepVariant** out) {
  static const SweepVariant r1[] = {
      variant<PolResid, TbCfg<PolResid, 1, 4, 16, 5, 1>>(),
      variant<PolResid, TbCfg<PolResid, 1, 2, 16, 5, 1>>(),
      variant<PolResid, TbCfg<PolResid, 1, 4, 8, 5, 2>>(),
      variant<PolResid, TbCfg<PolResid, 1, 8, 4, 4, 3>>(),
  };
  *out = r1;
  return sizeof(r1) / sizeof(r1[0]);
}

}  // namespace stencil
