// placeholder replaced by the request scheduler
#include "lp_runtime.h"
void lp_serve_shutdown(lp_ctx*) {}
