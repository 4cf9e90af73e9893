// The column-layout search kernel with iMBE's L - L' removal (Section II-C,
// embedded pruning): the same source as mbe_search.cu, compiled as its own
// translation unit (bitset level sets only).
#define MBE_PRUNE 1
#include "mbe_search.cu"
