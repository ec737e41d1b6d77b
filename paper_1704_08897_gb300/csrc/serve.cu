// Serving loop (continuous batching); filled in below the core solve path.
#include "../../include/biharm_ext.h"
