// lym1_pol_mixf.cu -- every kernel of the LYM1_MIXED_FAST policy.
#define LYM1_POL lym1::Policy<float, float, float, false>
#define LYM1_POL_NS pol_mixf
#include "lym1_pol_unit.cuh"
