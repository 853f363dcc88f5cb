// rn_file.cpp -- graph files: the engine's binary edge-list format (.rng) and the DIMACS
// shortest-path text format (.gr) in which road networks are commonly distributed.
//
// .rng, little-endian:
//   bytes 0-3   magic "RNG1"
//   u32         n (nodes)
//   u32         flags (RN_UNDIRECTED | RN_REORDER, as given to rn_graph_load)
//   u64         m (edges)
//   u32[m]      src, then u32[m] dst, then u32[m] w
// .gr (DIMACS): "c ..." comment lines, one "p sp n m" line, then m lines "a u v w" with
// 1-based node ids; every line is one arc (road files list both directions of a two-way
// road), read with flags RN_REORDER.
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>

#include "rn_internal.h"

namespace rn {

namespace {

struct File {
    std::FILE *f = nullptr;
    ~File() {
        if (f) std::fclose(f);
    }
};

constexpr char MAGIC[4] = {'R', 'N', 'G', '1'};

void read_exact(std::FILE *f, void *p, size_t bytes, const std::string &path) {
    if (bytes && std::fread(p, 1, bytes, f) != bytes) fail(RN_EINVAL, path + ": truncated file");
}

void read_rng(std::FILE *f, const std::string &path, EdgeFile *out) {
    uint32_t n = 0, flags = 0;
    uint64_t m = 0;
    read_exact(f, &n, 4, path);
    read_exact(f, &flags, 4, path);
    read_exact(f, &m, 8, path);
    if (flags & ~(RN_UNDIRECTED | RN_REORDER)) fail(RN_EINVAL, path + ": unknown flags in the header");
    // the arrays must be exactly what the header announces
    const long here = std::ftell(f);
    std::fseek(f, 0, SEEK_END);
    const long end = std::ftell(f);
    std::fseek(f, here, SEEK_SET);
    if (here < 0 || end < 0 || uint64_t(end - here) != 12 * m) fail(RN_EINVAL, path + ": size does not match m");
    out->n = n;
    out->flags = flags;
    out->src.resize(m);
    out->dst.resize(m);
    out->w.resize(m);
    read_exact(f, out->src.data(), 4 * m, path);
    read_exact(f, out->dst.data(), 4 * m, path);
    read_exact(f, out->w.data(), 4 * m, path);
}

void read_gr(std::FILE *f, const std::string &path, EdgeFile *out) {
    char line[512];
    uint64_t m = 0, arcs = 0, lineno = 0;
    bool header = false;
    while (std::fgets(line, sizeof line, f)) {
        lineno++;
        const std::string where = path + ":" + std::to_string(lineno);
        if (!std::strchr(line, '\n') && !std::feof(f)) fail(RN_EINVAL, where + ": line too long");
        if (line[0] == 'c' || line[0] == '\n' || line[0] == '\r' || line[0] == '\0') continue;
        if (line[0] == 'p') {
            unsigned long long n = 0, mm = 0;
            char kind[16] = {0};
            if (header || std::sscanf(line, "p %15s %llu %llu", kind, &n, &mm) != 3 || std::strcmp(kind, "sp") != 0 ||
                n >= 0xFFFFFFFFull)
                fail(RN_EINVAL, where + ": expected one 'p sp n m' line");
            out->n = uint32_t(n);
            m = mm;
            out->src.reserve(m);
            out->dst.reserve(m);
            out->w.reserve(m);
            header = true;
            continue;
        }
        if (line[0] == 'a') {
            unsigned long long u = 0, v = 0, w = 0;
            if (!header || std::sscanf(line, "a %llu %llu %llu", &u, &v, &w) != 3)
                fail(RN_EINVAL, where + ": expected 'a u v w' after the 'p' line");
            if (u < 1 || v < 1 || u > out->n || v > out->n) fail(RN_EINVAL, where + ": node id outside 1..n");
            if (w > 0xFFFFFFFFull) fail(RN_EINVAL, where + ": weight does not fit 32 bits");
            out->src.push_back(uint32_t(u - 1));
            out->dst.push_back(uint32_t(v - 1));
            out->w.push_back(uint32_t(w));
            arcs++;
            continue;
        }
        fail(RN_EINVAL, where + ": unknown line");
    }
    if (!header) fail(RN_EINVAL, path + ": no 'p sp n m' line");
    if (arcs != m) fail(RN_EINVAL, path + ": " + std::to_string(arcs) + " arcs, the header says " + std::to_string(m));
    out->flags = RN_REORDER;
}

}  // namespace

void read_edge_file(const char *path, EdgeFile *out) {
    if (!path) fail(RN_EINVAL, "null path");
    File f;
    f.f = std::fopen(path, "rb");
    if (!f.f) fail(RN_EINVAL, std::string(path) + ": cannot open");
    char magic[4] = {0};
    const size_t got = std::fread(magic, 1, 4, f.f);
    *out = EdgeFile{};
    if (got == 4 && std::memcmp(magic, MAGIC, 4) == 0) {
        read_rng(f.f, path, out);
    } else {
        std::rewind(f.f);
        read_gr(f.f, path, out);
    }
}

void write_edge_file(const char *path, uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                     const uint32_t *w, uint32_t flags) {
    if (!path) fail(RN_EINVAL, "null path");
    if (m && (!src || !dst || !w)) fail(RN_EINVAL, "null edge arrays with m > 0");
    if (flags & ~(RN_UNDIRECTED | RN_REORDER)) fail(RN_EINVAL, "unknown flag");
    File f;
    f.f = std::fopen(path, "wb");
    if (!f.f) fail(RN_EINVAL, std::string(path) + ": cannot create");
    bool ok = std::fwrite(MAGIC, 1, 4, f.f) == 4 && std::fwrite(&n, 4, 1, f.f) == 1 &&
              std::fwrite(&flags, 4, 1, f.f) == 1 && std::fwrite(&m, 8, 1, f.f) == 1;
    for (const uint32_t *a : {src, dst, w})
        ok = ok && (m == 0 || std::fwrite(a, 4, m, f.f) == m);
    ok = std::fclose(f.f) == 0 && ok;
    f.f = nullptr;
    if (!ok) fail(RN_EINVAL, std::string(path) + ": write failed");
}

}  // namespace rn
