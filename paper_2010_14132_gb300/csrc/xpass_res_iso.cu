// The dx == dy instances of the sweep's residual x-pass (see xpass_res.cu), in a
// translation unit of their own so that they compile in parallel with the others.
#define PGB_XRES_ISO 1
#include "xpass_res.cu"
