// Search kernels (single-CTA, batched, cooperative) for FCC cells.
#define HEA_SEARCH_KIND kFCC
#define HEA_SEARCH_LAUNCH launch_search_fcc
#define HEA_SEARCH_BATCH_LAUNCH launch_search_batch_fcc
#define HEA_COOP_LAUNCH launch_search_coop_fcc
#define HEA_COOP_MAXCTAS coop_max_ctas_fcc
#include "hea_search_kind.inc"
