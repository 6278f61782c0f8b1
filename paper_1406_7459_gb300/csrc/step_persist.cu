// step_persist.cu -- instantiations of the persistent Euler step for square
// power-of-two films (nx = ny = 64, 128, 256 with nz = 4; 256 x 256 with
// nz = 1, 2), its launch and the grid barrier's counters.
#include "step_persist.cuh"

namespace mmk {

template <int N, int NZ, int R>
static void fill_persist(PersistFns* f) {
    using Lay = PersistLayout<N, NZ, N, R>;
    f->k = k_step_persist<N, NZ, N, R>;
    f->t = Lay::T;
    f->smem = Lay::BYTES;
}

bool persist_lookup(int nx, int ny, int nz, int R, PersistFns* f) {
    if (nx != ny || R != 4) return false;
    if (nz == 4) {
        switch (nx) {
            case 64: fill_persist<64, 4, 4>(f); return true;
            case 128: fill_persist<128, 4, 4>(f); return true;
            case 256: fill_persist<256, 4, 4>(f); return true;
            default: return false;
        }
    }
    if (nx == 256 && nz == 2) {
        fill_persist<256, 2, 4>(f);
        return true;
    }
    if (nx == 256 && nz == 1) {
        fill_persist<256, 1, 4>(f);
        return true;
    }
    return false;
}

// Shared-memory attribute, and the grid: one block per plane and per tile,
// all co-resident (else the persistent step is not offered).
cudaError_t persist_configure(const Geom& g, int R, PersistFns* f, bool* usable) {
    *usable = false;
    cudaError_t e = cudaFuncSetAttribute(f->k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f->smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f->k, f->t, f->smem);
    if (e != cudaSuccess) return e;
    const int tiles = g.nz * (g.ny / R);
    f->grid = g.Hx > tiles ? g.Hx : tiles;
    *usable = per_sm >= 1 && (long long)per_sm * sms >= f->grid;
    return cudaSuccess;
}

cudaError_t persist_alloc_bar(GridBar** gb) {
    cudaError_t e = cudaMalloc(gb, sizeof(GridBar));
    if (e == cudaSuccess) e = cudaMemset(*gb, 0, sizeof(GridBar));
    return e;
}

cudaError_t launch_persist(const Geom& g, const PersistFns& f, const LlgCoef& c, const float* Kd, float2* S,
                           float2* Sh, const float* Min, float* Mout, int n, int* flag, GridBar* gb, long long limit,
                           cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(f.grid);
    cfg.blockDim = dim3(f.t);
    cfg.dynamicSmemBytes = f.smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, f.k, g, c, Kd, S, Sh, Min, Mout, n, flag, gb, limit);
}

}  // namespace mmk
