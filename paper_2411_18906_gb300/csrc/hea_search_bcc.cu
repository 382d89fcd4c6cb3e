// Single-CTA and batched search kernels for BCC cells.
#define HEA_SEARCH_KIND kBCC
#define HEA_PART_CHAIN
#define HEA_SEARCH_LAUNCH launch_search_bcc
#define HEA_SEARCH_BATCH_LAUNCH launch_search_batch_bcc
#include "hea_search_kind.inc"
