// method=direct (direct.cu): banded LU with partial pivoting on the device.
#pragma once

#include "common.cuh"

struct BandInfo {
    int64_t kl = 0, ku = 0;      // lower and upper bandwidth of the input
};

// x = A^{-1} b for a square CSR A (device), b and x device vectors of n.
// SS_ERR_UNSUPPORTED when the band does not fit; SS_ZERO_PIVOT for a singular A.
ss_status band_lu_solve(ss_ctx ctx, const DeviceCSR& A, const double2* b, double2* x, BandInfo* info);
