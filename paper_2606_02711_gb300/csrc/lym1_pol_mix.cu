// lym1_pol_mix.cu -- every kernel of the LYM1_MIXED policy.
#define LYM1_POL lym1::Policy<float, float, double, false>
#define LYM1_POL_NS pol_mix
#include "lym1_pol_unit.cuh"
