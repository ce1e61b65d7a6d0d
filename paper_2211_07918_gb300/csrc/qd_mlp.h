// Learned cost model (qd_mlp.cu): shapes shared with the planner.
#pragma once

namespace qd {
constexpr int kMlpIn = 12;      // launch features (qd_fuse.h)
constexpr int kMlpHidden = 64;  // three hidden layers of 64 ReLU units
constexpr int kMlpParams = kMlpIn * kMlpHidden + kMlpHidden + 2 * (kMlpHidden * kMlpHidden + kMlpHidden) +
                           kMlpHidden + 1;  // 9,217
}  // namespace qd
