// server.cu -- placeholder translation unit for the serving loop (filled in below).
#include "runtime.cuh"
void h3d_destroy_extras(heat3d_ctx*) {}
