// lym1_pol_f64.cu -- every kernel of the LYM1_FP64 policy.
#define LYM1_POL lym1::Policy<double, double, double, false>
#define LYM1_POL_NS pol_f64
#include "lym1_pol_unit.cuh"
