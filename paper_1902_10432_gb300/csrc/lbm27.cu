// D3Q27 instantiation of the lattice-Boltzmann kernels (namespace cbl::q27): the velocity set the
// paper prints (Sec. 3.2.1).
#define CBL_Q 27
#include "lbm.cu"
