// Cooperative search kernels for FCC cells.
#define HEA_SEARCH_KIND kFCC
#define HEA_PART_COOP
#define HEA_COOP_LAUNCH launch_search_coop_fcc
#define HEA_COOP_MAXCTAS coop_max_ctas_fcc
#include "hea_search_kind.inc"
