// The column-layout search kernel with the sorted-list path for level sets
// wider than the bitset limit (mbe_list.cuh): the same source as
// mbe_search.cu, compiled as its own translation unit.
#define MBE_LIST_PATH 1
#include "mbe_search.cu"
