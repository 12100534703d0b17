// Pool CTA kernel, rank bucket 16.
#define ISVD_TICK_KB 16
#include "pool_tick_inst.cuh"
