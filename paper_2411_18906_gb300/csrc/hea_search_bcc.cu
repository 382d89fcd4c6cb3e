// Search kernels (single-CTA, batched, cooperative) for BCC cells.
#define HEA_SEARCH_KIND kBCC
#define HEA_SEARCH_LAUNCH launch_search_bcc
#define HEA_SEARCH_BATCH_LAUNCH launch_search_batch_bcc
#define HEA_COOP_LAUNCH launch_search_coop_bcc
#define HEA_COOP_MAXCTAS coop_max_ctas_bcc
#include "hea_search_kind.inc"
