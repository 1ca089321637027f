// One edge update of the device CSR (Sec. 4: every insertion or deletion is
// one graph change, and the next update -- its effective resistance, its
// conditioned walks -- runs on the changed graph).  The edit keeps the layout
// every kernel reads: rows contiguous, each sorted strictly ascending (the
// neighbour index of the random-walk contract), row_off[n] = 2m.
//
// Insert (u, v), a = min(u, v), b = max(u, v): b enters row a at its sorted
// position pa and a enters row b at pb (old indices).  The new column array is
//     new[i] = old[i]      i <  pa
//     new[pa] = b
//     new[i] = old[i - 1]  pa < i <= pb      (row b's start moved by one)
//     new[pb + 1] = a
//     new[i] = old[i - 2]  i >  pb + 1
// Delete (u, v): pa and pb are the positions of b in row a and of a in row b,
//     new[i] = old[i]      i <  pa
//     new[i] = old[i + 1]  pa <= i < pb - 1
//     new[i] = old[i + 2]  i >= pb - 1
// and row_off[x] moves by +-([x > a] + [x > b]).  The columns are written to a
// scratch array and copied back, so the CSR keeps its device address (kernels
// and captured graphs that hold it stay valid).
#include "kc_common.cuh"

namespace kc {
namespace {

// pos[0] = pa, pos[1] = pb, pos[2] = error (1: the edit does not apply)
__global__ void k_edit_positions(const int64_t *row_off, const int32_t *col, int32_t a,
                                 int32_t b, int insert, int64_t *pos) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t p[2];
    bool ok = true;
    for (int k = 0; k < 2; ++k) {
        const int32_t row = k == 0 ? a : b, key = k == 0 ? b : a;
        int64_t lo = row_off[row], hi = row_off[row + 1];  // first index with col >= key
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (col[mid] < key) lo = mid + 1; else hi = mid;
        }
        const bool present = lo < row_off[row + 1] && col[lo] == key;
        if (present == (insert != 0)) ok = false;
        p[k] = lo;
    }
    pos[0] = p[0];
    pos[1] = p[1];
    pos[2] = ok ? 0 : 1;
}

__global__ void k_edit_cols(const int32_t *__restrict__ col, int32_t *__restrict__ out,
                            int64_t old_len, int64_t new_len, int32_t a, int32_t b, int insert,
                            const int64_t *__restrict__ pos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= new_len) return;
    if (pos[2]) {  // the edit does not apply: copy the old columns back unchanged
        out[i] = i < old_len ? col[i] : 0;
        return;
    }
    const int64_t pa = pos[0], pb = pos[1];
    int32_t x;
    if (insert) {
        if (i < pa) x = col[i];
        else if (i == pa) x = b;
        else if (i <= pb) x = col[i - 1];
        else if (i == pb + 1) x = a;
        else x = col[i - 2];
    } else {
        if (i < pa) x = col[i];
        else if (i < pb - 1) x = col[i + 1];
        else x = col[i + 2];
    }
    out[i] = x;
}

__global__ void k_edit_offsets(int64_t n, int64_t *row_off, int32_t a, int32_t b, int insert,
                               const int64_t *__restrict__ pos) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x > n || pos[2]) return;
    const int64_t d = (int64_t)(x > a) + (int64_t)(x > b);
    row_off[x] += insert ? d : -d;
}

}  // namespace

// Insert or delete the undirected edge (u, v) of an n-vertex CSR whose column
// array holds 2m entries now (capacity >= 2m + 2 for an insert).  `scratch`
// holds >= 2m + 2 int32 and `pos` 3 int64 of device memory.  Enqueued on s; a
// precondition failure (edge present on insert, absent on delete) leaves the
// CSR unchanged and pos[2] = 1.
cudaError_t launch_csr_edit(int64_t n, int64_t twom, int64_t *row_off, int32_t *col,
                            int32_t *scratch, int64_t *pos, int32_t u, int32_t v, bool insert,
                            cudaStream_t s) {
    const int32_t a = u < v ? u : v, b = u < v ? v : u;
    const int ins = insert ? 1 : 0;
    k_edit_positions<<<1, 32, 0, s>>>(row_off, col, a, b, ins, pos);
    const int64_t new_len = insert ? twom + 2 : twom - 2;
    if (new_len > 0) {
        k_edit_cols<<<(unsigned)((new_len + 255) / 256), 256, 0, s>>>(col, scratch, twom, new_len,
                                                                      a, b, ins, pos);
        cudaError_t e = cudaMemcpyAsync(col, scratch, sizeof(int32_t) * (size_t)new_len,
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    k_edit_offsets<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(n, row_off, a, b, ins, pos);
    return cudaGetLastError();
}

}  // namespace kc
