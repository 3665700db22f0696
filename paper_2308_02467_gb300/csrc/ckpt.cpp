// Element-network checkpoint file: a versioned little-endian binary with a CRC-32 trailer.
//
//   offset  size  field
//   0       8     magic "ELRTNET\0"
//   8       4     u32 version (2)
//   12      4     i32 p
//   16      4     i32 n_angles
//   20      4     i32 n_hidden
//   24      4     i32 width
//   28      4     i32 activation (0 GELU, 1 ELU)
//   32      8     u64 seed of the initial weights
//   40      4     i32 standardised (1 once elrt_net_fit has set the input/output standardisation)
//   44      8     i64 Adam step counter
//   52      8     i64 number F of FP32 values that follow
//   60      4     i32 input features (0 log kappa_hat, 1 kappa_hat)
//   64      4F    FP32 values (IEEE-754 bit patterns, little-endian), in this order:
//                 per layer l = 0 .. n_hidden: W [out][in_pad], b [out], Adam m and v of W, m and v of b;
//                 then the input mean and standard deviation [in_pad], the output mean and standard
//                 deviation [n_out]
//   64+4F   4     u32 CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320, initial value and final
//                 XOR 0xFFFFFFFF) of every byte before it
// The layout depends only on the description: in_pad = n_feat rounded up to 64 for layer 0 and
// width otherwise; out = width for hidden layers and n_out for the output layer (sizes as in
// elrt_net_sizes).  This file holds the host side: CRC, encoding and validation; no CUDA call.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "elrt_internal.h"

namespace {

const unsigned char kMagic[8] = {'E', 'L', 'R', 'T', 'N', 'E', 'T', 0};
constexpr uint32_t kVersion = 2;
constexpr size_t kHeaderBytes = 64;

uint32_t crc_table_entry(uint32_t c) {
    for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
    return c;
}

struct CrcTable {
    uint32_t t[256];
    CrcTable() {
        for (uint32_t i = 0; i < 256; ++i) t[i] = crc_table_entry(i);
    }
};

void put_u32(unsigned char* b, uint32_t v) {
    for (int i = 0; i < 4; ++i) b[i] = (unsigned char)(v >> (8 * i));
}
void put_u64(unsigned char* b, uint64_t v) {
    for (int i = 0; i < 8; ++i) b[i] = (unsigned char)(v >> (8 * i));
}
uint32_t get_u32(const unsigned char* b) {
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= (uint32_t)b[i] << (8 * i);
    return v;
}
uint64_t get_u64(const unsigned char* b) {
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v |= (uint64_t)b[i] << (8 * i);
    return v;
}

bool host_little_endian() {
    const uint32_t one = 1;
    unsigned char c;
    memcpy(&c, &one, 1);
    return c == 1;
}

// FP32 values <-> little-endian bytes
void floats_to_le(const float* src, size_t n, unsigned char* dst) {
    if (host_little_endian()) {
        memcpy(dst, src, n * 4);
        return;
    }
    for (size_t i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, src + i, 4);
        put_u32(dst + 4 * i, u);
    }
}
void le_to_floats(const unsigned char* src, size_t n, float* dst) {
    if (host_little_endian()) {
        memcpy(dst, src, n * 4);
        return;
    }
    for (size_t i = 0; i < n; ++i) {
        const uint32_t u = get_u32(src + 4 * i);
        memcpy(dst + i, &u, 4);
    }
}

}  // namespace

uint32_t ckpt_crc32(const void* data, size_t n, uint32_t crc) {
    static const CrcTable tab;
    const unsigned char* p = (const unsigned char*)data;
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) crc = tab.t[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return ~crc;
}

std::vector<size_t> ckpt_layout(const elrt_net_desc& d) {
    const int n1 = d.p + 1, nm = n1 * n1, nin = 2 * n1 * d.n_angles;
    const size_t fpad = (size_t)((nm + 1 + 63) / 64) * 64;
    const size_t nout = (size_t)nin * nin + (size_t)nm * nin;
    std::vector<size_t> v;
    const int nl = d.n_hidden + 1;
    for (int l = 0; l < nl; ++l) {
        const size_t in_pad = l == 0 ? fpad : (size_t)d.width;
        const size_t out = l == nl - 1 ? nout : (size_t)d.width;
        v.push_back(out * in_pad);  // W
        v.push_back(out);           // b
        v.push_back(out * in_pad);  // m of W
        v.push_back(out * in_pad);  // v of W
        v.push_back(out);           // m of b
        v.push_back(out);           // v of b
    }
    v.push_back(fpad);
    v.push_back(fpad);
    v.push_back(nout);
    v.push_back(nout);
    return v;
}

static bool desc_ok(const elrt_net_desc& d) {
    return d.p >= 1 && d.p <= 10 && d.n_angles >= 4 && d.n_angles <= 32 && d.n_angles % 4 == 0 && d.n_hidden >= 0 &&
           d.n_hidden <= 8 && d.width >= 64 && d.width % 64 == 0 && (d.activation == 0 || d.activation == 1) &&
           (d.features == 0 || d.features == 1);
}

bool ckpt_write(const char* path, const elrt_net_desc& d, int32_t standardised, int64_t step,
                const std::vector<const float*>& arrays, std::string* err) {
    const std::vector<size_t> lay = ckpt_layout(d);
    if (arrays.size() != lay.size()) {
        *err = "checkpoint: wrong number of arrays";
        return false;
    }
    size_t nf = 0;
    for (size_t c : lay) nf += c;
    unsigned char h[kHeaderBytes];
    memcpy(h, kMagic, 8);
    put_u32(h + 8, kVersion);
    put_u32(h + 12, (uint32_t)d.p);
    put_u32(h + 16, (uint32_t)d.n_angles);
    put_u32(h + 20, (uint32_t)d.n_hidden);
    put_u32(h + 24, (uint32_t)d.width);
    put_u32(h + 28, (uint32_t)d.activation);
    put_u64(h + 32, d.seed);
    put_u32(h + 40, (uint32_t)standardised);
    put_u64(h + 44, (uint64_t)step);
    put_u64(h + 52, (uint64_t)nf);
    put_u32(h + 60, (uint32_t)d.features);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) {
        *err = std::string("checkpoint: cannot open ") + tmp;
        return false;
    }
    bool ok = fwrite(h, 1, kHeaderBytes, f) == kHeaderBytes;
    uint32_t crc = ckpt_crc32(h, kHeaderBytes, 0);
    std::vector<unsigned char> buf;
    for (size_t a = 0; a < lay.size() && ok; ++a) {
        buf.resize(lay[a] * 4);
        floats_to_le(arrays[a], lay[a], buf.data());
        crc = ckpt_crc32(buf.data(), buf.size(), crc);
        ok = fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    }
    unsigned char t[4];
    put_u32(t, crc);
    ok = ok && fwrite(t, 1, 4, f) == 4;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        *err = std::string("checkpoint: write failed: ") + path;
        return false;
    }
    return true;
}

// Reads and validates the header (and, if payload != nullptr, the FP32 values); the CRC is always
// checked over the whole file.
bool ckpt_read(const char* path, elrt_net_desc* d, int32_t* standardised, int64_t* step, int64_t* n_floats,
               std::vector<float>* payload, std::string* err) {
    FILE* f = fopen(path, "rb");
    if (!f) {
        *err = std::string("checkpoint: cannot open ") + path;
        return false;
    }
    unsigned char h[kHeaderBytes];
    bool ok = fread(h, 1, kHeaderBytes, f) == kHeaderBytes;
    if (!ok || memcmp(h, kMagic, 8) != 0) {
        fclose(f);
        *err = "checkpoint: not an element-network checkpoint";
        return false;
    }
    if (get_u32(h + 8) != kVersion) {
        fclose(f);
        *err = "checkpoint: unsupported version";
        return false;
    }
    elrt_net_desc dd{};
    dd.p = (int32_t)get_u32(h + 12);
    dd.n_angles = (int32_t)get_u32(h + 16);
    dd.n_hidden = (int32_t)get_u32(h + 20);
    dd.width = (int32_t)get_u32(h + 24);
    dd.activation = (int32_t)get_u32(h + 28);
    dd.seed = get_u64(h + 32);
    const int32_t st = (int32_t)get_u32(h + 40);
    const int64_t sp = (int64_t)get_u64(h + 44);
    const uint64_t nf = get_u64(h + 52);
    dd.features = (int32_t)get_u32(h + 60);
    if (!desc_ok(dd) || (st != 0 && st != 1) || sp < 0) {
        fclose(f);
        *err = "checkpoint: invalid header";
        return false;
    }
    size_t expect = 0;
    for (size_t c : ckpt_layout(dd)) expect += c;
    if (nf != expect) {
        fclose(f);
        *err = "checkpoint: value count does not match the network description";
        return false;
    }
    uint32_t crc = ckpt_crc32(h, kHeaderBytes, 0);
    if (payload) payload->resize(expect);
    std::vector<unsigned char> buf(1 << 22);
    size_t done = 0;
    while (ok && done < expect) {
        const size_t take = std::min(buf.size() / 4, expect - done);
        ok = fread(buf.data(), 1, take * 4, f) == take * 4;
        if (!ok) break;
        crc = ckpt_crc32(buf.data(), take * 4, crc);
        if (payload) le_to_floats(buf.data(), take, payload->data() + done);
        done += take;
    }
    unsigned char t[4];
    ok = ok && fread(t, 1, 4, f) == 4;
    unsigned char extra;
    const bool at_end = ok && fread(&extra, 1, 1, f) == 0;
    fclose(f);
    if (!ok || !at_end) {
        *err = "checkpoint: truncated or oversized file";
        return false;
    }
    if (get_u32(t) != crc) {
        *err = "checkpoint: CRC mismatch";
        return false;
    }
    if (d) *d = dd;
    if (standardised) *standardised = st;
    if (step) *step = sp;
    if (n_floats) *n_floats = (int64_t)expect;
    return true;
}

extern "C" elrt_status elrt_net_file_info(const char* path, elrt_net_desc* desc, int32_t* standardised,
                                          int64_t* step, int64_t* n_values) {
    if (!path) return ELRT_EINVAL;
    std::string err;
    return ckpt_read(path, desc, standardised, step, n_values, nullptr, &err) ? ELRT_OK : ELRT_EINVAL;
}
