// Batched small-state kernels (filled in below).
#include "small.h"
