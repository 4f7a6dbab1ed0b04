// Lane capacity 48.
#define TSP_LMAX 48
#include "tsp_mlem_inst.cuh"
