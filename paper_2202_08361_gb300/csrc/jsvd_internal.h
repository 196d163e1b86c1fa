// jsvd_internal.h -- declarations shared between the library's .cu files.
#pragma once
#include "jsvd.h"

namespace jsvd {
int evd2_set_launch(int block, int blocks_per_sm);
}  // namespace jsvd
