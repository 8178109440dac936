// Plan files: a HostPlan and the point coordinates it was built from, in a
// plain binary layout (magic, version, then every field in a fixed order:
// scalars and arrays of scalars as raw bytes, structs field by field so that
// no padding byte is written, vectors as a 64-bit length followed by their
// elements, then a 64-bit FNV-1a checksum of the fields).  The same plan
// always gives the same file.  Loading rebuilds the device tables (and the transfer spectra)
// from these, skipping the octree, traversals and schedules.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include <sys/stat.h>
#include <unistd.h>

#include "plan.h"

namespace defmm {

namespace {

constexpr char kMagic[8] = {'D', 'E', 'F', 'M', 'M', 'P', 'L', 'N'};
constexpr uint32_t kVersion = 3;   // 2: Levels field by field (no padding bytes); 3: radial power

// 64-bit FNV-1a over every byte after the header, stored at the end of the
// file: a damaged plan file is refused instead of handing the kernels
// inconsistent tables.
struct Fnv1a {
    uint64_t h = 0xcbf29ce484222325ull;
    void add(const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 0x100000001b3ull; }
    }
};

struct Writer {
    FILE* f;
    Fnv1a sum;
    void bytes(const void* p, size_t n) {
        if (n && std::fwrite(p, 1, n, f) != n) throw std::runtime_error("plan file: write failed");
        sum.add(p, n);
    }
    template <typename V> void raw(const V& v) {
        static_assert(std::is_trivially_copyable<V>::value, "raw field");
        bytes(&v, sizeof(V));
    }
    template <typename V> void vec(const std::vector<V>& v) {
        static_assert(std::is_trivially_copyable<V>::value, "vector of raw elements");
        const uint64_t n = v.size();
        raw(n);
        bytes(v.data(), n * sizeof(V));
    }
    template <typename V> void vecvec(const std::vector<std::vector<V>>& v) {
        const uint64_t n = v.size();
        raw(n);
        for (const auto& x : v) vec(x);
    }
};

struct Reader {
    FILE* f;
    uint64_t left;   // bytes of the file not yet read
    Fnv1a sum;
    void bytes(void* p, size_t n) {
        if (n > left || (n && std::fread(p, 1, n, f) != n)) throw std::runtime_error("plan file: truncated");
        left -= n;
        sum.add(p, n);
    }
    template <typename V> void raw(V& v) {
        static_assert(std::is_trivially_copyable<V>::value, "raw field");
        bytes(&v, sizeof(V));
    }
    template <typename V> void vec(std::vector<V>& v) {
        uint64_t n = 0;
        raw(n);
        if (n > left / sizeof(V)) throw std::runtime_error("plan file: truncated");   // before allocating
        v.resize(n);
        bytes(v.data(), n * sizeof(V));
    }
    template <typename V> void vecvec(std::vector<std::vector<V>>& v) {
        uint64_t n = 0;
        raw(n);
        if (n > left / sizeof(uint64_t)) throw std::runtime_error("plan file: truncated");
        v.resize(n);
        for (auto& x : v) vec(x);
    }
};

// level ranges as two plain vectors (std::pair is not trivially copyable)
void level_ranges(Writer& w, const Tree& t) {
    std::vector<int32_t> a, b;
    for (const auto& r : t.level_range) { a.push_back(r.first); b.push_back(r.second); }
    w.vec(a); w.vec(b);
}
void level_ranges(Reader& r, Tree& t) {
    std::vector<int32_t> a, b;
    r.vec(a); r.vec(b);
    if (a.size() != b.size()) throw std::runtime_error("plan file: corrupt level ranges");
    t.level_range.clear();
    for (size_t i = 0; i < a.size(); ++i) t.level_range.emplace_back(a[i], b[i]);
}

template <typename A, typename T> void tree_fields(A& a, T& t) {
    a.vec(t.perm); a.vec(t.level); a.vec(t.ix); a.vec(t.iy); a.vec(t.iz);
    a.vec(t.begin); a.vec(t.end); a.vec(t.parent); a.vec(t.first_child); a.vec(t.nchild);
    level_ranges(a, t);
}

// Every HostPlan field, in one order for writing and reading.
template <typename A, typename H> void plan_fields(A& a, H& h) {
    a.raw(h.nx); a.raw(h.ny); a.raw(h.same); a.raw(h.kappa); a.raw(h.damping); a.raw(h.radial_power);
    a.raw(h.p); a.raw(h.N); a.raw(h.NF); a.raw(h.NFpad); a.raw(h.P3);
    a.raw(h.eta); a.raw(h.hf_kw); a.raw(h.self_eps_rel); a.raw(h.eps_self); a.raw(h.d_aabb); a.raw(h.side);
    a.raw(h.corner);
    a.raw(h.lv.side0); a.raw(h.lv.kappa); a.raw(h.lv.eta); a.raw(h.lv.hf_kw); a.raw(h.lv.hf); a.raw(h.lv.l_hf);
    tree_fields(a, h.tt);
    tree_fields(a, h.ts_own);
    a.vec(h.m2l); a.vec(h.p2p); a.vecvec(h.marks_t); a.vecvec(h.marks_s);
    a.vec(h.m_cell); a.vec(h.m_dir); a.vec(h.m_first); a.vec(h.m_count);
    a.vec(h.l_cell); a.vec(h.l_dir); a.vec(h.l_first); a.vec(h.l_count);
    a.vec(h.m_slot); a.vec(h.l_slot);
    a.vec(h.slot_level); a.vec(h.slot_dir); a.vec(h.slot_u); a.vec(h.slot_P); a.vec(h.slot_Q);
    a.vec(h.m1); a.vec(h.tw);
    a.vec(h.spec_level); a.vec(h.spec_kbar);
    a.vec(h.m2f_list); a.vec(h.mhat_of_m);
    a.vec(h.grp_member_off); a.vec(h.grp_members); a.vec(h.grp_chunk_off); a.vec(h.grp_half);
    a.vec(h.chk_blk_off); a.vec(h.chk_nspec); a.vec(h.chk_blk); a.vec(h.chk_op_off); a.vec(h.chk_op);
    a.raw(h.chk_max_blocks); a.raw(h.chk_stage_blocks);
    a.vecvec(h.m2m_lvl); a.vecvec(h.l2l_lvl); a.vecvec(h.l2l_par);
    a.vec(h.p2m_cells); a.vec(h.l2p_cells);
    a.vec(h.p2p_unit_leaf); a.vec(h.p2p_unit_off); a.vec(h.p2p_sbeg); a.vec(h.p2p_send); a.vec(h.p2p_soff);
    a.vec(h.p2p_part); a.vec(h.p2p_leaf); a.vec(h.p2p_leaf_off); a.vec(h.p2p_leaf_units);
    a.raw(h.p2p_parts); a.raw(h.p2p_interactions);
    a.raw(h.ngeo);
    a.vec(h.geo_point_off); a.vec(h.geo_cell_off); a.vec(h.geo_level_off);
    a.vec(h.geo_kappa); a.vec(h.geo_eps); a.vec(h.geo_center);
    a.vec(h.level_side_u); a.vec(h.cell_corner_u); a.vec(h.cell_geo); a.vec(h.spec_kappa);
}

}  // namespace

void save_plan_file(const std::string& path, const HostPlan& hp, const std::vector<double>& X,
                    const std::vector<double>& Y) {
    // A regular (or new) file is written under a temporary name in the same
    // directory and renamed over `path` once complete, so a failed save leaves
    // neither a partial file nor a damaged earlier one.  Anything else (a
    // device, a pipe) is written in place and never renamed or removed.
    struct stat st;
    const bool in_place = ::stat(path.c_str(), &st) == 0 && !S_ISREG(st.st_mode);
    const std::string tmp = in_place ? path : path + ".tmp" + std::to_string((long)::getpid());
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) throw std::runtime_error("plan file: cannot open " + path + " for writing");
    try {
        Writer w{f, {}};
        w.raw(kMagic);
        w.raw(kVersion);
        w.sum = Fnv1a{};
        plan_fields(w, hp);
        w.vec(X);
        w.vec(Y);
        const uint64_t h = w.sum.h;
        w.raw(h);
    } catch (...) {
        std::fclose(f);
        if (!in_place) std::remove(tmp.c_str());
        throw;
    }
    if (std::fclose(f) != 0) {
        if (!in_place) std::remove(tmp.c_str());
        throw std::runtime_error("plan file: write failed");
    }
    if (!in_place && std::rename(tmp.c_str(), path.c_str()) != 0) {
        std::remove(tmp.c_str());
        throw std::runtime_error("plan file: cannot rename the written file to " + path);
    }
}

void load_plan_file(const std::string& path, HostPlan& hp, std::vector<double>& X, std::vector<double>& Y) {
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f) throw std::runtime_error("plan file: cannot open " + path);
    try {
        if (std::fseek(f, 0, SEEK_END) != 0) throw std::runtime_error("plan file: cannot seek " + path);
        const long size = std::ftell(f);
        if (size < 0 || std::fseek(f, 0, SEEK_SET) != 0) throw std::runtime_error("plan file: cannot seek " + path);
        Reader r{f, (uint64_t)size, {}};
        char magic[8];
        uint32_t version = 0;
        r.raw(magic);
        if (std::memcmp(magic, kMagic, 8) != 0) throw std::runtime_error("plan file: not a defmm plan");
        r.raw(version);
        if (version != kVersion) throw std::runtime_error("plan file: unsupported version");
        r.sum = Fnv1a{};
        plan_fields(r, hp);
        r.vec(X);
        r.vec(Y);
        const uint64_t h = r.sum.h;
        uint64_t stored = 0;
        r.raw(stored);
        if (stored != h || r.left != 0) throw std::runtime_error("plan file: checksum mismatch (damaged file)");
        if ((int64_t)X.size() != 3 * hp.nx || (!hp.same && (int64_t)Y.size() != 3 * hp.ny))
            throw std::runtime_error("plan file: coordinates do not match the plan");
    } catch (...) {
        std::fclose(f);
        throw;
    }
    std::fclose(f);
}

}  // namespace defmm
