// Cooperative search kernels for BCC cells.
#define HEA_SEARCH_KIND kBCC
#define HEA_PART_COOP
#define HEA_COOP_LAUNCH launch_search_coop_bcc
#define HEA_COOP_MAXCTAS coop_max_ctas_bcc
#include "hea_search_kind.inc"
