// checkpoint.cu -- ct_factor_save / ct_factor_load: a factorisation written
// to a file and read back, so A = QR is computed once per geometry and reused
// across runs (the paper's reuse of Eq. 2 for every system sharing A).
//
// File layout (little-endian): FileHeader, then VR column by column (M' x n,
// no leading-dimension padding), tau[n], T blocks (nblocks x NB x NB), V tops
// (nblocks x NB x NB); elements in the factor's storage type.  The header
// carries an FNV-1a 64-bit checksum of the header itself (with the checksum
// field zeroed) followed by everything after it, and a loader accepts block
// sizes only in the form the factorisation produces them.
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>

#include "handles.cuh"

namespace ctqr {
namespace {

constexpr char kMagic[8] = {'C', 'T', 'Q', 'R', 'F', 'A', 'C', '1'};
constexpr uint32_t kVersion = 4;  // 2: fan-beam geometry fields; 3: projector; 4: header checksummed
constexpr size_t kChunk = (size_t)64 << 20;

struct FileHeader {
    char magic[8];
    uint32_t version;
    int32_t precision;
    int64_t M, n, m, nb_outer, nb_inner, nblocks;
    ct_geometry geom;
    double rjj_min, rjj_max;
    uint64_t checksum;
};

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n) {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
};

struct PinnedBuf {
    void *p = nullptr;
    ~PinnedBuf() {
        if (p) cudaFreeHost(p);
    }
};

bool same_geom(const ct_geometry &a, const ct_geometry &b) {
    return a.n_side == b.n_side && a.n_views == b.n_views && a.n_bins == b.n_bins &&
           a.pixel_width == b.pixel_width && a.bin_width == b.bin_width && a.arc_deg == b.arc_deg &&
           a.sqrt_lambda == b.sqrt_lambda && a.kind == b.kind && a.source_dist == b.source_dist &&
           a.fan_deg == b.fan_deg && a.projector == b.projector;
}

// Device regions of a factor in file order: (pointer, rows, cols, ld).
struct Region {
    void *dev;
    int64_t rows, cols, ld;
};

// Block sizes as ct_qr_factor / ct_qr_factor_ooc make them: panel width nb in
// [1, 32], outer width NB a multiple of both nb and 32, and one T / V-top
// block per NB columns.  Anything else would index T and the V tops past their
// allocations in the solve.
bool blocks_valid(const FileHeader &hd) {
    return hd.nb_inner >= 1 && hd.nb_inner <= 32 && hd.nb_outer >= 32 && hd.nb_outer <= (1 << 15) &&
           hd.nb_outer % 32 == 0 && hd.nb_outer % hd.nb_inner == 0 && hd.n > 0 &&
           hd.nblocks == ceil_div(hd.n, hd.nb_outer);
}

// Hash of the header with its checksum field zeroed.
void hash_header(Fnv &fnv, const FileHeader &hd) {
    unsigned char b[sizeof(FileHeader)];
    memcpy(b, &hd, sizeof(hd));  // bytes as written, padding included
    memset(b + offsetof(FileHeader, checksum), 0, sizeof(hd.checksum));
    fnv.add(b, sizeof(b));
}

int regions(ct_factor f, Region *out) {
    out[0] = {f->ooc ? f->VR_host : f->VR, f->M, f->n, f->lda};  // host memory for out-of-core factors
    out[1] = {f->tau, f->n, 1, f->n};
    out[2] = {f->Tall, (int64_t)f->NB * f->NB, f->nblocks, (int64_t)f->NB * f->NB};
    out[3] = {f->Vtop, (int64_t)f->NB * f->NB, f->nblocks, (int64_t)f->NB * f->NB};
    return 4;
}

}  // namespace
}  // namespace ctqr

using namespace ctqr;

extern "C" ct_status ct_factor_save(ct_factor f, const char *path) {
    if (!f || !path || !f->sys) return CT_ERR_ARG;
    if (f->store) {
        set_error("a disk-resident factor is its own checkpoint: reopen its file with "
                  "ct_system_open_disk and call ct_qr_factor_ooc");
        return CT_ERR_UNSUPPORTED;
    }
    FILE *fp = fopen(path, "wb");
    if (!fp) {
        set_error("cannot open %s for writing", path);
        return CT_ERR_ARG;
    }
    FileHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, kMagic, 8);
    hd.version = kVersion;
    hd.precision = (int32_t)f->prec;
    hd.M = f->M;
    hd.n = f->n;
    hd.m = f->m;
    hd.nb_outer = f->NB;
    hd.nb_inner = f->nb;
    hd.nblocks = f->nblocks;
    hd.geom = f->sys->geom;
    hd.rjj_min = f->rjj_min;
    hd.rjj_max = f->rjj_max;
    ct_status st = CT_OK;
    PinnedBuf buf;
    Fnv fnv;
    hash_header(fnv, hd);
    if (fwrite(&hd, sizeof(hd), 1, fp) != 1) st = CT_ERR_ARG;
    if (st == CT_OK && cudaMallocHost(&buf.p, kChunk) != cudaSuccess) st = CT_ERR_HOSTMEM;
    const size_t es = f->es();
    Region rg[4];
    const int nr = regions(f, rg);
    for (int r = 0; r < nr && st == CT_OK; ++r) {
        const int64_t cols_per = std::max<int64_t>(1, (int64_t)(kChunk / (es * rg[r].rows)));
        for (int64_t c0 = 0; c0 < rg[r].cols && st == CT_OK; c0 += cols_per) {
            const int64_t nc = std::min(cols_per, rg[r].cols - c0);
            const size_t rb = es * rg[r].rows;
            if (cudaMemcpy2D(buf.p, rb, (char *)rg[r].dev + es * rg[r].ld * c0, es * rg[r].ld, rb, nc,
                             cudaMemcpyDefault) != cudaSuccess) {
                st = CT_ERR_CUDA;
                break;
            }
            fnv.add(buf.p, rb * nc);
            if (fwrite(buf.p, rb, nc, fp) != (size_t)nc) st = CT_ERR_ARG;
        }
    }
    if (st == CT_OK) {
        hd.checksum = fnv.h;
        if (fseek(fp, 0, SEEK_SET) != 0 || fwrite(&hd, sizeof(hd), 1, fp) != 1) st = CT_ERR_ARG;
    }
    if (fclose(fp) != 0 && st == CT_OK) st = CT_ERR_ARG;
    if (st != CT_OK) set_error("writing factor checkpoint %s failed (%s)", path, ct_status_str(st));
    return st;
}

extern "C" ct_status ct_factor_load(ct_system sys, const char *path, void *stream, ct_factor *out) {
    if (!sys || !path || !out) return CT_ERR_ARG;
    *out = nullptr;
    FILE *fp = fopen(path, "rb");
    if (!fp) {
        set_error("cannot open %s", path);
        return CT_ERR_ARG;
    }
    FileHeader hd;
    if (fread(&hd, sizeof(hd), 1, fp) != 1 || memcmp(hd.magic, kMagic, 8) != 0 ||
        hd.version != kVersion) {
        fclose(fp);
        set_error("%s is not a factor checkpoint of this version", path);
        return CT_ERR_ARG;
    }
    const bool fp64 = hd.precision == CT_FP64;
    if (!same_geom(hd.geom, sys->geom) || fp64 != sys->fp64 || hd.M != sys->rows || hd.n != sys->n ||
        hd.m != sys->m || hd.precision < CT_FP64 || hd.precision > CT_BF16X3_REFINE) {
        fclose(fp);
        set_error("checkpoint %s does not match this system's geometry/precision", path);
        return CT_ERR_ARG;
    }
    if (!blocks_valid(hd)) {
        fclose(fp);
        set_error("checkpoint %s has invalid block sizes (nb_outer %lld, nb_inner %lld, %lld blocks)",
                  path, (long long)hd.nb_outer, (long long)hd.nb_inner, (long long)hd.nblocks);
        return CT_ERR_ARG;
    }
    ct_factor f = new (std::nothrow) ct_factor_s;
    if (!f) {
        fclose(fp);
        return CT_ERR_HOSTMEM;
    }
    f->sys = sys;
    f->prec = (ct_precision)hd.precision;
    f->fp64 = fp64;
    f->kind = solve_kind(f->prec);
    f->upd_kind = update_kind(f->prec);
    f->M = hd.M;
    f->n = hd.n;
    f->m = hd.m;
    f->lda = sys->lda;
    f->NB = (int)hd.nb_outer;
    f->nb = (int)hd.nb_inner;
    f->nblocks = hd.nblocks;
    f->rjj_min = hd.rjj_min;
    f->rjj_max = hd.rjj_max;
    const size_t es = f->es();
    ct_status st = CT_OK;
    // VR overwrites the system's dense storage, as a factorisation would; a
    // system whose storage already went to another factor gets a fresh one.
    bool took_dense = false;
    if (sys->dense) {
        f->VR = sys->dense;
        sys->dense = nullptr;
        took_dense = true;
    } else if (cudaMalloc(&f->VR, es * (size_t)f->lda * f->n) != cudaSuccess) {
        st = CT_ERR_OOM;
    }
    f->Rm = f->VR;
    f->ldr = f->lda;
    if (st == CT_OK && !took_dense && f->lda > f->M &&
        cudaMemsetAsync(f->VR, 0, es * (size_t)f->lda * f->n, (cudaStream_t)stream) != cudaSuccess)
        st = CT_ERR_CUDA;
    if (st != CT_OK ||
        cudaMalloc(&f->tau, es * (size_t)f->n) != cudaSuccess ||
        cudaMalloc(&f->Tall, es * (size_t)f->nblocks * f->NB * f->NB) != cudaSuccess ||
        cudaMalloc(&f->Vtop, es * (size_t)f->nblocks * f->NB * f->NB) != cudaSuccess)
        st = st == CT_OK ? CT_ERR_OOM : st;
    PinnedBuf buf;
    Fnv fnv;
    hash_header(fnv, hd);
    if (st == CT_OK && cudaMallocHost(&buf.p, kChunk) != cudaSuccess) st = CT_ERR_HOSTMEM;
    if (st == CT_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) st = CT_ERR_CUDA;
    Region rg[4];
    const int nr = regions(f, rg);
    for (int r = 0; r < nr && st == CT_OK; ++r) {
        const int64_t cols_per = std::max<int64_t>(1, (int64_t)(kChunk / (es * rg[r].rows)));
        for (int64_t c0 = 0; c0 < rg[r].cols && st == CT_OK; c0 += cols_per) {
            const int64_t nc = std::min(cols_per, rg[r].cols - c0);
            const size_t rb = es * rg[r].rows;
            if (fread(buf.p, rb, nc, fp) != (size_t)nc) {
                st = CT_ERR_ARG;
                break;
            }
            fnv.add(buf.p, rb * nc);
            if (cudaMemcpy2D((char *)rg[r].dev + es * rg[r].ld * c0, es * rg[r].ld, buf.p, rb, rb, nc,
                             cudaMemcpyHostToDevice) != cudaSuccess)
                st = CT_ERR_CUDA;
        }
    }
    fclose(fp);
    if (st == CT_OK && fnv.h != hd.checksum) st = CT_ERR_ARG;
    if (st != CT_OK) {
        set_error("reading factor checkpoint %s failed (%s)", path, ct_status_str(st));
        if (took_dense) {  // hand the storage back (its content is no longer A~)
            sys->dense = f->VR;
            f->VR = nullptr;
        }
        ct_factor_free(f);
        return st;
    }
    *out = f;
    return CT_OK;
}
