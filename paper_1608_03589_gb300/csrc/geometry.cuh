// Pixel-tile geometry of the direct kernels (internal): tile and stage sizes and the
// per-angle coordinate table.  Kept apart from the other shared declarations so that the
// direct kernels' sources can be identified by their own files.
#pragma once

namespace bp {

// Direct kernels work on square pixel tiles; the per-angle table below gives the
// detector coordinate u (in bins) of pixel (0,0) and its change per tile, in 32.32
// fixed point (exact integer tile stepping), plus the per-pixel steps in float.
constexpr int kTile = 64;         // pixel tile side of the direct R* / R kernels
constexpr int kStage = 16;        // angles per shared-memory stage
constexpr int kThreads = 256;     // threads per CTA of the direct kernels

struct AngleParam {
    long long U00;  // u(pixel 0,0) * 2^32
    long long CT;   // u step per tile along x (kTile pixels) * 2^32
    long long ST;   // u step per tile along y * 2^32
    float c;        // u step per pixel along x = cos(theta) dx/dt
    float s;        // u step per pixel along y = sin(theta) dx/dt
    float w;        // quadrature weight w_k
    float pad;
};
static_assert(sizeof(AngleParam) == 40, "AngleParam layout");

}  // namespace bp
