// Lane capacity 12.
#define TSP_LMAX 12
#include "tsp_mlem_inst.cuh"
