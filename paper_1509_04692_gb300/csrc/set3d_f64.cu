// 3D set-kernel instantiations (set3d_f64); filled in with the 3D sweep.
#include "hpmc_launch.h"
