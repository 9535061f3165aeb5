// Batched persistent kernels: many element sets of uneven size and mixed
// type/kind. Each block repeatedly takes the next tile of its combination from a
// global counter and runs the same tile code as the single-set kernels; nothing
// waits on another block. Tiles are implicit (BatchSeg): the tile index gives the
// item by binary search over the combination's segment table.
#include "fe_kernels.cuh"

namespace fe {

template <int COMBO> struct ComboCfg;
#define FE_COMBO(ID, ET, KD, Q, CP, TP)                                          \
    template <> struct ComboCfg<ID> {                                            \
        static constexpr int et = ET, kind = KD, quad = Q, cpq = CP, tpe = TP;   \
    };
FE_COMBO(0, TET, POISSON, Q_TET1, 0, 1)
FE_COMBO(1, TET, POISSON, Q_TET1, 1, 1)
FE_COMBO(2, TET, POISSON, Q_TET4, 0, 1)
FE_COMBO(3, TET, POISSON, Q_TET4, 1, 1)
FE_COMBO(4, TET, GENERIC, Q_TET1, 0, 1)
FE_COMBO(5, TET, GENERIC, Q_TET1, 1, 1)
FE_COMBO(6, TET, GENERIC, Q_TET4, 0, 1)
FE_COMBO(7, TET, GENERIC, Q_TET4, 1, 1)
FE_COMBO(8, PRISM, POISSON, Q_PRISM6, 0, 1)
FE_COMBO(9, PRISM, POISSON, Q_PRISM6, 1, 1)
FE_COMBO(10, PRISM, GENERIC, Q_PRISM6, 0, 1)
FE_COMBO(11, PRISM, GENERIC, Q_PRISM6, 1, 1)
FE_COMBO(12, PRISM, POISSON, Q_PRISM6, 0, 2)
FE_COMBO(13, PRISM, POISSON, Q_PRISM6, 1, 2)
FE_COMBO(14, PRISM, GENERIC, Q_PRISM6, 0, 2)
FE_COMBO(15, PRISM, GENERIC, Q_PRISM6, 1, 2)
#undef FE_COMBO

template <int ID>
__device__ __forceinline__ bool tile_combo(const BatchItemDev *item, long long first, int count, unsigned char *smem,
                                           uint64_t *bar, unsigned *phase) {
    using K = ComboCfg<ID>;
    const ElemParams p = item->p;
    return process_tile<K::et, K::kind, MIXED, K::quad, K::cpq, AOS, AOS, K::tpe>(p, first, count, smem, bar,
                                                                                   *phase);
}

template <int ID> __device__ __forceinline__ void fix_combo(const ElemParams &p, int64_t e) {
    using K = ComboCfg<ID>;
    fixup_element<K::et, K::kind, MIXED, K::quad, K::cpq, AOS, AOS>(p, e);
}

// Next tile of a combination for one thread: counter, then the item by binary
// search over the segment table (segs[0].first_tile == 0).
struct TileRef {
    unsigned t, item;
    long long first;
    int count;
};
template <int ID>
__device__ __forceinline__ TileRef find_tile(unsigned t, const BatchItemDev *items, unsigned n_items,
                                             const BatchSeg *segs, unsigned n_segs, unsigned n_tiles, int B) {
    TileRef r{t, 0xFFFFFFFFu, 0, 0};
    if (r.t < n_tiles && n_segs > 0) {
        unsigned lo = 0, hi = n_segs;
        while (hi - lo > 1) {
            const unsigned mid = (lo + hi) >> 1;
            if (segs[mid].first_tile <= r.t) lo = mid;
            else hi = mid;
        }
        const BatchSeg sg = segs[lo];
        r.first = static_cast<long long>(r.t - sg.first_tile) * B;
        if (sg.item < n_items && r.first < sg.n && items[sg.item].combo == ID) {
            r.item = sg.item;
            const long long left = sg.n - r.first;
            r.count = left < B ? int(left) : B;
        }
    }
    return r;
}
template <int ID>
__device__ __forceinline__ TileRef next_tile(const BatchItemDev *items, unsigned n_items, const BatchSeg *segs,
                                             unsigned n_segs, unsigned n_tiles, unsigned *tile_counter, int B) {
    return find_tile<ID>(atomicAdd(tile_counter, 1u), items, n_items, segs, n_segs, n_tiles, B);
}

// Kernel of one combination. Persistent (tile_counter given): blocks take the
// next tile of this combination from its counter until none is left; one lane
// of warp 1 looks up the following tile while the block loads and computes the
// current one (double-buffered in shared memory), so the counter and the search
// stay off the block's critical path. Without a counter: block b takes tiles b,
// b + gridDim.x, ... (a grid of one block per tile), so that the hardware block
// scheduler overlaps one block's stores with the next block's loads. A batch
// launches one such kernel per combination present (one register allocation per
// combination).
template <int ID>
__global__ void __launch_bounds__(256) batch_kernel(const BatchItemDev *__restrict__ items, unsigned n_items,
                                                    const BatchSeg *__restrict__ segs, unsigned n_segs, unsigned n_tiles,
                                                    unsigned *tile_counter, int *status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ TileRef s_ref[2];
    const int B = blockDim.x / ComboCfg<ID>::tpe;                 // elements per tile
    const int R = blockDim.x > 32 ? 32 : 0;  // the looking-up thread (not the copy issuer, thread 0)
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    unsigned phase = 0;
    if (!tile_counter) {
        for (unsigned t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            if (threadIdx.x == R) s_ref[0] = find_tile<ID>(t, items, n_items, segs, n_segs, n_tiles, B);
            __syncthreads();
            const TileRef cur = s_ref[0];
            if (cur.item == 0xFFFFFFFFu) {
                if (threadIdx.x == 0) atomicOr(status, ST_BAD_TILE);
                __syncthreads();
                continue;
            }
            if (!tile_combo<ID>(items + cur.item, cur.first, cur.count, smem, &bar, &phase)) return;
        }
        if (threadIdx.x < 32) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        return;
    }
    if (threadIdx.x == R) s_ref[0] = next_tile<ID>(items, n_items, segs, n_segs, n_tiles, tile_counter, B);
    __syncthreads();
    for (unsigned i = 0;; ++i) {
        const TileRef cur = s_ref[i & 1u];
        if (cur.t >= n_tiles) break;
        // s_ref[(i + 1) & 1] was last read at the start of iteration i - 1, before
        // the barriers of that tile
        if (threadIdx.x == R) s_ref[(i + 1) & 1u] = next_tile<ID>(items, n_items, segs, n_segs, n_tiles, tile_counter, B);
        if (cur.item == 0xFFFFFFFFu) {
            if (threadIdx.x == 0) atomicOr(status, ST_BAD_TILE);
            __syncthreads();
            continue;
        }
        if (!tile_combo<ID>(items + cur.item, cur.first, cur.count, smem, &bar, &phase)) return;
    }
    if (threadIdx.x < 32) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Fix-up of every flagged element of the batch (list entries: item << 40 | element).
__global__ void __launch_bounds__(256) batch_fixup_kernel(const BatchItemDev *__restrict__ items, unsigned n_items,
                                                          const unsigned long long *__restrict__ list,
                                                          const unsigned *count, unsigned cap, int *status) {
    const unsigned c = *count;
    const unsigned n = c < cap ? c : cap;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long ent = list[i];
        const unsigned item = static_cast<unsigned>(ent >> 40);
        const int64_t e = static_cast<int64_t>(ent & ((1ull << 40) - 1));
        if (item >= n_items || e >= items[item].p.n) {
            atomicOr(status, ST_BAD_TILE);
            continue;
        }
        const ElemParams p = items[item].p;
        switch (items[item].combo) {
            case 0: fix_combo<0>(p, e); break;
            case 1: fix_combo<1>(p, e); break;
            case 2: fix_combo<2>(p, e); break;
            case 3: fix_combo<3>(p, e); break;
            case 4: fix_combo<4>(p, e); break;
            case 5: fix_combo<5>(p, e); break;
            case 6: fix_combo<6>(p, e); break;
            case 7: fix_combo<7>(p, e); break;
            case 8: fix_combo<8>(p, e); break;
            case 9: fix_combo<9>(p, e); break;
            case 10: fix_combo<10>(p, e); break;
            case 11: fix_combo<11>(p, e); break;
            case 12: fix_combo<12>(p, e); break;
            case 13: fix_combo<13>(p, e); break;
            case 14: fix_combo<14>(p, e); break;
            case 15: fix_combo<15>(p, e); break;
            default: atomicOr(status, ST_BAD_TILE); break;
        }
    }
}

template <int ID> static long long smem_of(int B) {
    using K = ComboCfg<ID>;
    return BlockSmem<K::et, K::kind, MIXED, K::quad, K::cpq>::total(B);
}

long long batch_smem_bytes(int combo, int B) {
    switch (combo) {
        case 0: return smem_of<0>(B);
        case 1: return smem_of<1>(B);
        case 2: return smem_of<2>(B);
        case 3: return smem_of<3>(B);
        case 4: return smem_of<4>(B);
        case 5: return smem_of<5>(B);
        case 6: return smem_of<6>(B);
        case 7: return smem_of<7>(B);
        case 8: return smem_of<8>(B);
        case 9: return smem_of<9>(B);
        case 10: return smem_of<10>(B);
        case 11: return smem_of<11>(B);
        case 12: return smem_of<12>(B);
        case 13: return smem_of<13>(B);
        case 14: return smem_of<14>(B);
        case 15: return smem_of<15>(B);
    }
    return -1;
}

const void *kernel_batch(int combo) {
    switch (combo) {
        case 0: return reinterpret_cast<const void *>(&batch_kernel<0>);
        case 1: return reinterpret_cast<const void *>(&batch_kernel<1>);
        case 2: return reinterpret_cast<const void *>(&batch_kernel<2>);
        case 3: return reinterpret_cast<const void *>(&batch_kernel<3>);
        case 4: return reinterpret_cast<const void *>(&batch_kernel<4>);
        case 5: return reinterpret_cast<const void *>(&batch_kernel<5>);
        case 6: return reinterpret_cast<const void *>(&batch_kernel<6>);
        case 7: return reinterpret_cast<const void *>(&batch_kernel<7>);
        case 8: return reinterpret_cast<const void *>(&batch_kernel<8>);
        case 9: return reinterpret_cast<const void *>(&batch_kernel<9>);
        case 10: return reinterpret_cast<const void *>(&batch_kernel<10>);
        case 11: return reinterpret_cast<const void *>(&batch_kernel<11>);
        case 12: return reinterpret_cast<const void *>(&batch_kernel<12>);
        case 13: return reinterpret_cast<const void *>(&batch_kernel<13>);
        case 14: return reinterpret_cast<const void *>(&batch_kernel<14>);
        case 15: return reinterpret_cast<const void *>(&batch_kernel<15>);
    }
    return nullptr;
}
const void *kernel_batch_fixup() { return reinterpret_cast<const void *>(&batch_fixup_kernel); }

// Failure-detection self-test: one block arms its mbarrier for 16 bytes that no
// copy will ever deliver and waits with the same bounded loop as the tiles. The
// wait must give up after `polls` polls and record the timeout in the status
// word; nothing is in flight when the block exits.
__global__ void selftest_wait_kernel(unsigned polls, int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
    __syncthreads();
    mbar_wait_bounded(&bar, 0, status, polls);
}

const void *kernel_selftest_wait() { return reinterpret_cast<const void *>(&selftest_wait_kernel); }

}  // namespace fe
