// Lane capacity 24.
#define TSP_LMAX 24
#include "tsp_mlem_inst.cuh"
