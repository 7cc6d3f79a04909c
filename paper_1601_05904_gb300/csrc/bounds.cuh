// Index checks of the bounds-checked build (a substitute for a memory
// checker on GPUs where none can run).
//
// Built with -DAIDW_BOUNDS_CHECK (build(checked=True), libaidw_checked.so),
// AIDW_IN(i, n, site) tests 0 <= i < n; when the test fails it counts the
// violation in this translation unit's record, keeps the site and index of
// the first one, and yields false, so the access it guards is skipped (no
// trap, no out-of-range access).  aidw_bounds_report() adds up the records
// of all translation units.  In the normal build AIDW_IN is the constant
// true, its arguments are not evaluated, and the guarded code is unchanged.
#pragma once

#include <cuda_runtime.h>

namespace aidw {
namespace bounds {

// Where a check sits (the high 16 bits of a recorded violation).
enum Site : int {
    kKeyCell = 1,         // cell of a point or query, against the grid's cells
    kScatterHead = 2,     // cell head read by the scatter
    kScatterDest = 3,     // scatter destination, against the point (or query) count
    kFixupHead = 4,       // cell of a record in the fix-up, against the grid's cells
    kFixupSegment = 5,    // end of that cell's segment, against the point count
    kFixupDest = 6,       // stable destination, against the point count
    kKnnOrder = 7,        // query taken from the cell order, against the query count
    kKnnHead = 8,         // cell head of a ring segment, against the cells + 1
    kKnnPoints = 9,       // end of a ring segment's points, against the point count
    kWeightTile = 10,     // weighting tile of a unit, against the tiles of the grid
    kWeightPiece = 11,    // end of a unit's piece, against the tile length
    kTestHook = 12,       // aidw_test_bounds_check (no access behind it)
    kWeightSlot = 13,     // stream-K partial-sum slot, against the slots of the launch
};

// Reads one translation unit's record (count, first = site << 48 | index).
using Reader = void (*)(unsigned long long *count, unsigned long long *first);
bool add_reader(Reader r);  // api.cu: registers a translation unit's reader

#ifdef AIDW_BOUNDS_CHECK
static __device__ unsigned long long g_count = 0ull;
static __device__ unsigned long long g_first = ~0ull;

static __device__ __noinline__ bool fail(int site, long long i)
{
    atomicAdd(&g_count, 1ull);
    atomicCAS(&g_first, ~0ull,
              ((unsigned long long)site << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFull));
    return false;
}

static void read_record(unsigned long long *count, unsigned long long *first)
{
    unsigned long long c = 0, f = ~0ull;
    if (cudaMemcpyFromSymbol(&c, g_count, sizeof(c)) != cudaSuccess ||
        cudaMemcpyFromSymbol(&f, g_first, sizeof(f)) != cudaSuccess) {
        cudaGetLastError();
        c = 0;
        f = ~0ull;
    }
    *count = c;
    *first = f;
}
[[maybe_unused]] static const bool g_registered = add_reader(&read_record);
#endif

}  // namespace bounds
}  // namespace aidw

#ifdef AIDW_BOUNDS_CHECK
#define AIDW_IN(i, n, site)                                             \
    (((long long)(i) >= 0 && (long long)(i) < (long long)(n))           \
         ? true                                                         \
         : ::aidw::bounds::fail((site), (long long)(i)))
#else
#define AIDW_IN(i, n, site) true
#endif
