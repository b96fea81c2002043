// hierfile.cu -- a hierarchy and its boot triplets as one binary file
// (samg_export, samg_write_hierarchy, samg_import_file).  The paper has no
// file format; this is storage for the solve phase's inputs: the finest
// operator A, the interpolation operators P_l, Q_l (from which the Galerkin
// operators of Eq. coarseOp are rebuilt on import) and the boot triplets.
//
// Layout, little-endian, no padding:
//   "SAMGHIER" | u32 version (1) | u32 kind | u32 target | u32 n_b | u32 n_levels
//   csr A | for l < n_levels - 1: csr P_l, then csr Q_l (SVD kind only)
//   f64 sigma[n_b] | f64 U[rows_u][n_b] | f64 V[n][n_b] (SVD kind only)
//   u64 FNV-1a hash of every byte before it
// csr = i32 m | i32 n | i64 nnz | i64 row_ptr[m + 1] | i32 col[nnz] | f64 val[nnz]
// rows_u = m for the SVD kind, n for SPD_EIG.  Host code only.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hierfile.cuh"

namespace samg {

namespace {

constexpr char kMagic[8] = {'S', 'A', 'M', 'G', 'H', 'I', 'E', 'R'};
constexpr uint32_t kVersion = 1;

uint64_t fnv1a(const unsigned char *p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct Writer {
    std::vector<unsigned char> buf;
    template <typename T>
    void put(const T &v) {
        const unsigned char *p = reinterpret_cast<const unsigned char *>(&v);
        buf.insert(buf.end(), p, p + sizeof(T));
    }
    template <typename T>
    void put_n(const T *v, size_t n) {
        if (!n) return;
        const unsigned char *p = reinterpret_cast<const unsigned char *>(v);
        buf.insert(buf.end(), p, p + n * sizeof(T));
    }
    void csr(const HCsr &a) {
        put<int32_t>(a.m);
        put<int32_t>(a.n);
        put<int64_t>(a.nnz());
        put_n(a.rp.data(), a.rp.size());
        put_n(a.ci.data(), a.ci.size());
        put_n(a.v.data(), a.v.size());
    }
};

struct Reader {
    const unsigned char *p;
    size_t n, at = 0;
    void need(size_t bytes) const {
        SAMG_CHECK(bytes <= n - at, SAMG_E_INVALID, "hierarchy file: truncated");
    }
    template <typename T>
    T get() {
        need(sizeof(T));
        T v;
        std::memcpy(&v, p + at, sizeof(T));
        at += sizeof(T);
        return v;
    }
    template <typename T>
    void get_n(std::vector<T> &out, int64_t count) {
        SAMG_CHECK(count >= 0, SAMG_E_INVALID, "hierarchy file: negative count");
        // the size check comes before any allocation, so a corrupted count
        // cannot ask for more memory than the file could fill
        SAMG_CHECK((uint64_t)count <= (n - at) / sizeof(T), SAMG_E_INVALID, "hierarchy file: truncated");
        out.resize((size_t)count);
        if (count) std::memcpy(out.data(), p + at, (size_t)count * sizeof(T));
        at += (size_t)count * sizeof(T);
    }
    void csr(HCsr &a) {
        a.m = get<int32_t>();
        a.n = get<int32_t>();
        const int64_t nnz = get<int64_t>();
        SAMG_CHECK(a.m >= 0 && a.n >= 0 && nnz >= 0, SAMG_E_INVALID, "hierarchy file: negative size");
        get_n(a.rp, (int64_t)a.m + 1);
        get_n(a.ci, nnz);
        get_n(a.v, nnz);
    }
};

}  // namespace

void write_hierarchy_file(const std::string &path, const HierFile &h) {
    const bool spd = h.kind == SAMG_SPD_EIG;
    const int nlev = (int)h.P.size() + 1;
    SAMG_CHECK(nlev >= 2 && (spd || h.Q.size() == h.P.size()), SAMG_E_INVALID,
               "hierarchy file: need P (and Q) for every level but the coarsest");
    const size_t ru = (size_t)(spd ? h.A.n : h.A.m);
    SAMG_CHECK(h.sigma.size() == (size_t)h.nb && h.U.size() == ru * h.nb &&
                   (spd || h.V.size() == (size_t)h.A.n * h.nb),
               SAMG_E_INVALID, "hierarchy file: triplet sizes do not match A and n_b");
    Writer w;
    w.put_n(kMagic, 8);
    w.put<uint32_t>(kVersion);
    w.put<uint32_t>((uint32_t)h.kind);
    w.put<uint32_t>((uint32_t)h.target);
    w.put<uint32_t>((uint32_t)h.nb);
    w.put<uint32_t>((uint32_t)nlev);
    w.csr(h.A);
    for (int l = 0; l + 1 < nlev; ++l) {
        w.csr(h.P[l]);
        if (!spd) w.csr(h.Q[l]);
    }
    w.put_n(h.sigma.data(), h.sigma.size());
    w.put_n(h.U.data(), h.U.size());
    if (!spd) w.put_n(h.V.data(), h.V.size());
    w.put<uint64_t>(fnv1a(w.buf.data(), w.buf.size()));
    FILE *f = std::fopen(path.c_str(), "wb");
    SAMG_CHECK(f != nullptr, SAMG_E_INVALID, "hierarchy file: cannot open " + path + " for writing");
    const size_t put = std::fwrite(w.buf.data(), 1, w.buf.size(), f);
    const bool ok = std::fclose(f) == 0 && put == w.buf.size();
    SAMG_CHECK(ok, SAMG_E_INVALID, "hierarchy file: write to " + path + " failed");
}

void read_hierarchy_file(const std::string &path, HierFile &h) {
    FILE *f = std::fopen(path.c_str(), "rb");
    SAMG_CHECK(f != nullptr, SAMG_E_INVALID, "hierarchy file: cannot open " + path);
    std::vector<unsigned char> buf;
    unsigned char tmp[1 << 16];
    size_t got;
    while ((got = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + got);
    const bool err = std::ferror(f) != 0;
    std::fclose(f);
    SAMG_CHECK(!err, SAMG_E_INVALID, "hierarchy file: read of " + path + " failed");
    SAMG_CHECK(buf.size() >= 8 + 5 * 4 + 8 && std::memcmp(buf.data(), kMagic, 8) == 0, SAMG_E_INVALID,
               "hierarchy file: not a hierarchy file");
    uint64_t stored;
    std::memcpy(&stored, buf.data() + buf.size() - 8, 8);
    SAMG_CHECK(stored == fnv1a(buf.data(), buf.size() - 8), SAMG_E_INVALID,
               "hierarchy file: checksum mismatch (corrupted file)");
    Reader r{buf.data(), buf.size() - 8};
    r.at = 8;
    SAMG_CHECK(r.get<uint32_t>() == kVersion, SAMG_E_INVALID, "hierarchy file: unknown version");
    const uint32_t kind = r.get<uint32_t>(), target = r.get<uint32_t>();
    const uint32_t nb = r.get<uint32_t>(), nlev = r.get<uint32_t>();
    SAMG_CHECK(kind <= 1 && target <= 1 && nb >= 1 && nb <= 16 && nlev >= 2 && nlev <= 64,
               SAMG_E_INVALID, "hierarchy file: bad header fields");
    h.kind = (samg_kind)kind;
    h.target = (samg_target)target;
    h.nb = (int)nb;
    const bool spd = h.kind == SAMG_SPD_EIG;
    r.csr(h.A);
    h.P.assign(nlev - 1, HCsr());
    h.Q.assign(spd ? 0 : nlev - 1, HCsr());
    for (uint32_t l = 0; l + 1 < nlev; ++l) {
        r.csr(h.P[l]);
        if (!spd) r.csr(h.Q[l]);
    }
    r.get_n(h.sigma, (int64_t)nb);
    r.get_n(h.U, (int64_t)(spd ? h.A.n : h.A.m) * nb);
    if (spd) h.V.clear();
    else r.get_n(h.V, (int64_t)h.A.n * nb);
    SAMG_CHECK(r.at == r.n, SAMG_E_INVALID, "hierarchy file: trailing bytes");
}

}  // namespace samg
