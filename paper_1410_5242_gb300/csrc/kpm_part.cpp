// Row partition of the KPM-DOS problem for several processes (Sec.
// "Symmetric Heterogeneous Execution": each process holds a contiguous,
// weighted share of the rows; before every sweep it receives the entries
// of the vector block its rows read from other processes' rows, the halo;
// the scalar products are summed over processes once, at the end, as in the
// single global reduction of Table III).  Host only.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "kpm_internal.h"

extern "C" {

int kpm_partition_rows(int64_t n, int32_t parts, const double *weights, int64_t align,
                       int64_t *row_start)
{
    if (n < 1 || parts < 1 || align < 1 || !row_start || n % align != 0)
        return KPM_EINVAL;
    const int64_t units = n / align;  // whole planes
    if (units < parts)
        return KPM_EINVAL;
    double total = 0.0;
    for (int32_t k = 0; k < parts; k++) {
        const double w = weights ? weights[k] : 1.0;
        if (!(w > 0.0) || !std::isfinite(w))
            return KPM_EINVAL;
        total += w;
    }
    // boundary k at the rounded cumulative share, at least one plane per part
    double acc = 0.0;
    row_start[0] = 0;
    for (int32_t k = 1; k < parts; k++) {
        acc += weights ? weights[k - 1] : 1.0;
        int64_t u = (int64_t)std::llround(acc / total * (double)units);
        const int64_t lo = row_start[k - 1] / align + 1;  // one plane more than the last
        const int64_t hi = units - (parts - k);           // room for the parts after it
        u = std::min(std::max(u, lo), hi);
        row_start[k] = u * align;
    }
    row_start[parts] = n;
    return KPM_OK;
}

int kpm_partition_build(int64_t n, const int64_t *row_ptr, const int32_t *col,
                        const double *val_ri, int32_t parts, const int64_t *row_start,
                        int32_t part, kpm_part *out)
{
    if (!out)
        return KPM_EINVAL;
    std::memset(out, 0, sizeof(*out));
    if (parts < 1 || part < 0 || part >= parts || !row_start || row_start[0] != 0 ||
        row_start[parts] != n)
        return KPM_EINVAL;
    for (int32_t k = 0; k < parts; k++)
        if (row_start[k + 1] <= row_start[k])
            return KPM_EINVAL;
    int rc = kpm::validate_csr(n, row_ptr, col, val_ri);
    if (rc)
        return rc;
    auto owner = [&](int64_t row) {
        return (int32_t)(std::upper_bound(row_start, row_start + parts + 1, row) - row_start - 1);
    };
    const int64_t r0 = row_start[part], r1 = row_start[part + 1], n_loc = r1 - r0;
    try {
        // the halo: rows of other parts that this part's rows read, increasing
        std::vector<int64_t> halo;
        for (int64_t i = r0; i < r1; i++)
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
                if (col[k] < r0 || col[k] >= r1)
                    halo.push_back(col[k]);
        std::sort(halo.begin(), halo.end());
        halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
        // what the other parts read of this part's rows: for each part q, the
        // rows of [r0, r1) its entries reference, increasing (q's halo order)
        std::map<int32_t, std::vector<int32_t>> send;
        for (int32_t q = 0; q < parts; q++) {
            if (q == part)
                continue;
            std::vector<int32_t> rows;
            for (int64_t i = row_start[q]; i < row_start[q + 1]; i++)
                for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
                    if (col[k] >= r0 && col[k] < r1)
                        rows.push_back((int32_t)(col[k] - r0));
            std::sort(rows.begin(), rows.end());
            rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
            if (!rows.empty())
                send[q] = std::move(rows);
        }
        // peers: every part this one receives from or sends to, increasing
        std::vector<int32_t> peers;
        for (int64_t h : halo)
            peers.push_back(owner(h));
        for (auto &kv : send)
            peers.push_back(kv.first);
        std::sort(peers.begin(), peers.end());
        peers.erase(std::unique(peers.begin(), peers.end()), peers.end());

        const int64_t nnz = row_ptr[r1] - row_ptr[r0];
        const int np = (int)peers.size();
        int64_t n_send = 0;
        for (auto &kv : send)
            n_send += (int64_t)kv.second.size();
        out->n = n;
        out->row0 = r0;
        out->n_local = n_loc;
        out->n_halo = (int64_t)halo.size();
        out->nnz = nnz;
        out->n_peers = np;
        out->row_ptr = (int64_t *)std::malloc(sizeof(int64_t) * (n_loc + 1));
        out->col = (int32_t *)std::malloc(sizeof(int32_t) * (nnz ? nnz : 1));
        out->val_ri = (double *)std::malloc(sizeof(double) * 2 * (nnz ? nnz : 1));
        out->halo_rows = (int64_t *)std::malloc(sizeof(int64_t) * (halo.empty() ? 1 : halo.size()));
        out->peer = (int32_t *)std::malloc(sizeof(int32_t) * (np ? np : 1));
        out->recv_ptr = (int64_t *)std::malloc(sizeof(int64_t) * (np + 1));
        out->send_ptr = (int64_t *)std::malloc(sizeof(int64_t) * (np + 1));
        out->send_rows = (int32_t *)std::malloc(sizeof(int32_t) * (n_send ? n_send : 1));
        if (!out->row_ptr || !out->col || !out->val_ri || !out->halo_rows || !out->peer ||
            !out->recv_ptr || !out->send_ptr || !out->send_rows) {
            kpm_partition_release(out);
            return KPM_ENOMEM;
        }
        // local CSR: a column in [r0, r1) becomes its local row, another the
        // local row count plus its halo slot; within a row the local columns
        // stay increasing and come before the halo ones
        for (int64_t i = 0; i <= n_loc; i++)
            out->row_ptr[i] = row_ptr[r0 + i] - row_ptr[r0];
        for (int64_t i = r0; i < r1; i++) {
            std::vector<std::pair<int64_t, int64_t>> entries;  // (local column, source entry)
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
                const int64_t c = col[k];
                const int64_t lc = (c >= r0 && c < r1)
                                       ? c - r0
                                       : n_loc + (std::lower_bound(halo.begin(), halo.end(), c) -
                                                  halo.begin());
                entries.emplace_back(lc, k);
            }
            std::sort(entries.begin(), entries.end());
            int64_t at = out->row_ptr[i - r0];
            for (auto &e : entries) {
                out->col[at] = (int32_t)e.first;
                out->val_ri[2 * at] = val_ri[2 * e.second];
                out->val_ri[2 * at + 1] = val_ri[2 * e.second + 1];
                at++;
            }
        }
        std::copy(halo.begin(), halo.end(), out->halo_rows);
        out->recv_ptr[0] = out->send_ptr[0] = 0;
        for (int q = 0; q < np; q++) {
            out->peer[q] = peers[q];
            // halo slots owned by peer q: contiguous, the halo being increasing
            const int64_t lo = std::lower_bound(halo.begin(), halo.end(), row_start[peers[q]]) -
                               halo.begin();
            const int64_t hi = std::lower_bound(halo.begin(), halo.end(), row_start[peers[q] + 1]) -
                               halo.begin();
            (void)lo;
            out->recv_ptr[q + 1] = hi;
            const auto it = send.find(peers[q]);
            const int64_t cnt = it == send.end() ? 0 : (int64_t)it->second.size();
            if (cnt)
                std::copy(it->second.begin(), it->second.end(), out->send_rows + out->send_ptr[q]);
            out->send_ptr[q + 1] = out->send_ptr[q] + cnt;
        }
        return KPM_OK;
    } catch (const std::bad_alloc &) {
        kpm_partition_release(out);
        return KPM_ENOMEM;
    }
}

void kpm_partition_release(kpm_part *p)
{
    if (!p)
        return;
    std::free(p->row_ptr);
    std::free(p->col);
    std::free(p->val_ri);
    std::free(p->halo_rows);
    std::free(p->peer);
    std::free(p->recv_ptr);
    std::free(p->send_ptr);
    std::free(p->send_rows);
    std::memset(p, 0, sizeof(*p));
}

}  // extern "C"
