// Single-CTA and batched search kernels for FCC cells.
#define HEA_SEARCH_KIND kFCC
#define HEA_PART_CHAIN
#define HEA_SEARCH_LAUNCH launch_search_fcc
#define HEA_SEARCH_BATCH_LAUNCH launch_search_batch_fcc
#include "hea_search_kind.inc"
