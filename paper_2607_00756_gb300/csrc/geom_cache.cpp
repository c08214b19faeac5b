// On-disk cache of the host geometry: beams, parents and the FP64 Sibson
// weights (Algorithm 5's build steps; the weights depend only on the
// aperture, the detector and the rings, so they are computed once per
// such geometry and reused across runs).
//
// One file per geometry, named by a 64-bit FNV-1a hash of the bip_config
// fields the geometry reads.  The file repeats those fields, so a hash
// collision is detected, and ends with an FNV-1a checksum of its contents;
// a file that fails any check is ignored (counted as rejected) and
// rewritten.  Files are written to a temporary name and renamed into place,
// so a reader never sees a partial file.  The format is native-endian
// (both supported hosts, x86-64 and aarch64, are little-endian).
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <unistd.h>

#include "bip_internal.h"

namespace {

constexpr char kMagic[8] = {'B', 'I', 'P', 'G', 'E', 'O', 'M', 0};
constexpr uint32_t kVersion = 1;

std::mutex g_mu;
std::string g_dir;                       // empty: no cache
bool g_env_read = false;
std::atomic<int64_t> g_hits{0}, g_misses{0}, g_rejected{0};
std::atomic<uint64_t> g_tmp_seq{0};       // temporary file names unique within the process

uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

// The geometry's inputs, packed without padding so that hashing and
// comparing them is well defined.
struct KeyFields {
    int32_t i[13];
    double d[7];
};

KeyFields key_fields(const bip_config& c) {
    KeyFields k;
    std::memset(&k, 0, sizeof(k));
    const int32_t iv[13] = {c.ny, c.nx, c.fy, c.fx, c.nrad1, c.nang1, c.nrad2, c.nang2,
                            c.dfy, c.dfx, c.cube_ky, c.cube_kx, 0};
    const double dv[7] = {c.ly, c.lx, c.e0, c.alpha, c.theta_det, c.defocus, c.cs};
    std::memcpy(k.i, iv, sizeof(iv));
    std::memcpy(k.d, dv, sizeof(dv));
    return k;
}

uint64_t key_hash(const KeyFields& k) {
    uint64_t h = fnv1a(&kVersion, sizeof(kVersion));
    h = fnv1a(k.i, sizeof(k.i), h);
    return fnv1a(k.d, sizeof(k.d), h);
}

struct Writer {
    std::vector<unsigned char> buf;
    void raw(const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        buf.insert(buf.end(), b, b + n);
    }
    template <class T> void pod(const T& v) { raw(&v, sizeof(T)); }
    template <class T> void vec(const std::vector<T>& v) {
        const uint64_t n = v.size();
        pod(n);
        if (n) raw(v.data(), n * sizeof(T));
    }
};

struct Reader {
    const unsigned char* p;
    size_t left;
    bool ok = true;
    bool raw(void* out, size_t n) {
        if (!ok || n > left) return ok = false;
        std::memcpy(out, p, n);
        p += n;
        left -= n;
        return true;
    }
    template <class T> bool pod(T& v) { return raw(&v, sizeof(T)); }
    template <class T> bool vec(std::vector<T>& v, uint64_t max_elems) {
        uint64_t n = 0;
        if (!pod(n) || n > max_elems || n * sizeof(T) > left) return ok = false;
        v.resize(n);
        return n == 0 || raw(v.data(), n * sizeof(T));
    }
};

std::string dir_locked() {
    if (!g_env_read) {
        g_env_read = true;
        const char* e = std::getenv("BIP_GEOMETRY_CACHE");
        if (e && *e && g_dir.empty()) g_dir = e;
    }
    return g_dir;
}

std::string path_for(const std::string& dir, uint64_t key) {
    char name[64];
    std::snprintf(name, sizeof(name), "/bip-geometry-%016llx.bin", (unsigned long long)key);
    return dir + name;
}

void serialize(const KeyFields& k, uint64_t key, const BipGeometry& g, Writer& w) {
    w.raw(kMagic, sizeof(kMagic));
    w.pod(kVersion);
    w.pod(key);
    w.pod(k);
    w.pod(g.lambda);
    w.pod(g.sigma);
    w.pod(g.psi_norm);
    const int32_t iv[8] = {g.n_full, g.B, g.n_det, g.Bp1, g.Bp2, g.dfy, g.dfx, g.n_cube};
    w.raw(iv, sizeof(iv));
    w.vec(g.h_beam);
    w.vec(g.h_det);
    w.vec(g.h_cube);
    w.vec(g.p1);
    w.vec(g.p2);
    w.vec(g.w1);
    w.vec(g.w2);
    w.vec(g.psi_beam);
    const uint64_t sum = fnv1a(w.buf.data(), w.buf.size());
    w.pod(sum);
}

// Parses and checks a file's bytes; true only if everything is consistent.
bool deserialize(const std::vector<unsigned char>& bytes, const KeyFields& k, uint64_t key, BipGeometry& g) {
    if (bytes.size() < sizeof(kMagic) + sizeof(uint64_t)) return false;
    uint64_t sum = 0;
    std::memcpy(&sum, bytes.data() + bytes.size() - sizeof(sum), sizeof(sum));
    if (fnv1a(bytes.data(), bytes.size() - sizeof(sum)) != sum) return false;
    Reader r{bytes.data(), bytes.size() - sizeof(sum)};
    char magic[8];
    uint32_t version = 0;
    uint64_t fkey = 0;
    KeyFields fk;
    if (!r.raw(magic, sizeof(magic)) || std::memcmp(magic, kMagic, sizeof(kMagic)) != 0) return false;
    if (!r.pod(version) || version != kVersion) return false;
    if (!r.pod(fkey) || fkey != key) return false;
    if (!r.pod(fk) || std::memcmp(&fk, &k, sizeof(k)) != 0) return false;
    BipGeometry t;
    int32_t iv[8];
    if (!r.pod(t.lambda) || !r.pod(t.sigma) || !r.pod(t.psi_norm) || !r.raw(iv, sizeof(iv))) return false;
    t.n_full = iv[0];
    t.B = iv[1];
    t.n_det = iv[2];
    t.Bp1 = iv[3];
    t.Bp2 = iv[4];
    t.dfy = iv[5];
    t.dfx = iv[6];
    t.n_cube = iv[7];
    const uint64_t grid = (uint64_t)k.i[0] * (uint64_t)k.i[1];
    if (t.B <= 0 || t.n_det <= 0 || t.n_cube < 0 || t.Bp1 < 0 || t.Bp2 < 0 || (uint64_t)t.B > grid ||
        (uint64_t)t.n_det > grid || (uint64_t)t.n_cube > grid || t.Bp1 > t.B || t.Bp2 > t.n_det)
        return false;
    if (!r.vec(t.h_beam, 2 * grid) || !r.vec(t.h_det, 2 * grid) || !r.vec(t.h_cube, 2 * grid) ||
        !r.vec(t.p1, grid) || !r.vec(t.p2, grid) || !r.vec(t.w1, grid * grid) || !r.vec(t.w2, grid * grid) ||
        !r.vec(t.psi_beam, grid))
        return false;
    if (r.left != 0) return false;
    if (t.h_beam.size() != 2 * (size_t)t.B || t.h_det.size() != 2 * (size_t)t.n_det ||
        t.h_cube.size() != 2 * (size_t)t.n_cube || t.p1.size() != (size_t)t.Bp1 || t.p2.size() != (size_t)t.Bp2 ||
        t.w1.size() != (size_t)t.B * t.Bp1 || t.w2.size() != (size_t)t.n_det * t.Bp2 ||
        t.psi_beam.size() != (size_t)t.B)
        return false;
    for (int32_t p : t.p1)
        if (p < 0 || p >= t.B) return false;
    for (int32_t p : t.p2)
        if (p < 0 || p >= t.n_det) return false;
    g = std::move(t);
    return true;
}

bool read_file(const std::string& path, std::vector<unsigned char>& out) {
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f) return false;
    out.clear();
    unsigned char chunk[1 << 16];
    size_t n;
    while ((n = std::fread(chunk, 1, sizeof(chunk), f)) > 0) out.insert(out.end(), chunk, chunk + n);
    const bool ok = !std::ferror(f);
    std::fclose(f);
    return ok;
}

void write_file(const std::string& path, const std::vector<unsigned char>& bytes) {
    // unique per process and write, so concurrent writers (threads or
    // processes) never share a temporary file; the rename is atomic
    const std::string tmp = path + ".tmp." + std::to_string((long long)getpid()) + "." +
                            std::to_string((unsigned long long)++g_tmp_seq);
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;                      // an unwritable cache only costs the rebuild
    const bool ok = std::fwrite(bytes.data(), 1, bytes.size(), f) == bytes.size();
    const bool closed = std::fclose(f) == 0;
    if (ok && closed && std::rename(tmp.c_str(), path.c_str()) == 0) return;
    std::remove(tmp.c_str());
}

}  // namespace

bip_status bip_geometry_cached(const bip_config& cfg, BipGeometry& g, std::string& err) {
    std::string dir;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        dir = dir_locked();
    }
    if (dir.empty()) return bip_build_geometry(cfg, g, err);
    const KeyFields k = key_fields(cfg);
    const uint64_t key = key_hash(k);
    const std::string path = path_for(dir, key);
    std::vector<unsigned char> bytes;
    if (read_file(path, bytes)) {
        if (deserialize(bytes, k, key, g)) {
            ++g_hits;
            return BIP_OK;
        }
        ++g_rejected;
    }
    const bip_status st = bip_build_geometry(cfg, g, err);
    if (st != BIP_OK) return st;
    ++g_misses;
    Writer w;
    serialize(k, key, g, w);
    write_file(path, w.buf);
    return BIP_OK;
}

extern "C" {

bip_status bip_set_geometry_cache(const char* dir) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_env_read = true;                   // an explicit setting overrides BIP_GEOMETRY_CACHE
    g_dir = dir ? dir : "";
    while (g_dir.size() > 1 && g_dir.back() == '/') g_dir.pop_back();
    return BIP_OK;
}

bip_status bip_geometry_cache_stats(int64_t* hits, int64_t* misses, int64_t* rejected) {
    if (hits) *hits = g_hits.load();
    if (misses) *misses = g_misses.load();
    if (rejected) *rejected = g_rejected.load();
    return BIP_OK;
}

}  // extern "C"
