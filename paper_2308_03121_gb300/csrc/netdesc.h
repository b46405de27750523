// Network description ("nvisr-net 1") parser of the library.
//
// NNVISR consumes a network through a description of its graph plus weights
// (Section 3.1: networks arrive as exported graph files and are described by
// n and the Interpolation / Extra frame / Double frame flags).  This library
// reads a minimal text form of such a graph: per-layer statements with every
// activation, residual add, PixelShuffle and weight sharing explicit, and an
// FP32 weight blob in statement order (weight [cout][cin][k][k] then bias).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace nvisr {

struct NetLayer {
    std::string op;                  // "conv" | "dcn"
    std::string name;
    std::vector<std::string> in;     // sources (channel concatenation)
    std::string om;                  // dcn: offset/mask head tensor
    std::string add;                 // residual source (added after the activation)
    std::string share;               // layer whose weights are reused
    int cin = 0, cout = 0, k = 3, groups = 1, ps = 0, act = 0;
    // PixelShuffle factors (rows, columns): ps=r gives (r, r); psy= / psx= give them apart
    // (out[c, psy*h + i, psx*w + j] = in[c*psy*psx + i*psx + j, h, w]); (1, 1) = none
    int psy = 1, psx = 1;
    int64_t woff = -1;               // offset of weights in the blob (floats)
    int owner = -1;                  // index of the layer owning the weights
};

struct NetOutput {
    std::string name;
    std::vector<std::string> skip;   // frames whose upsampled mean is added
};

struct NetDesc {
    std::string family = "tuple";    // "tuple" | "group"
    int frames = 1;
    int scale = 1;                   // horizontal scale (the isotropic scale when scale_y equals it)
    int scale_y = 1;                 // vertical scale ("scale sx sy"; "scale s" sets both)
    int align = 1;
    bool interp = false, extra = false, dbl = false;
    int skip = 0;                    // 0 none, 1 nearest, 2 bilinear
    bool yuv = false;                // network domain: R'G'B' (default) or Y'CbCr (Section 3.1)
    std::vector<NetLayer> layers;
    std::vector<NetOutput> outputs;
    int64_t weights_used = 0;
    int find(const std::string &name) const;
};

// Parses text; checks shapes, sources, sharing and that the blob holds
// exactly the floats the layers use.  Returns false with a message on error.
bool parse_netdesc(const char *text, int64_t blob_count, NetDesc *out, std::string *err);

}  // namespace nvisr
