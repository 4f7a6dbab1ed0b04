// Lane capacity 64.
#define TSP_LMAX 64
#include "tsp_mlem_inst.cuh"
