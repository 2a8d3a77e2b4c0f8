// codec.h -- internal interface of the 8-bit log depth codec (codec.cu) for
// the lift kernel: the decode table of IMLOC_DEPTH_LOG8 views.
#pragma once

namespace imloc {

constexpr int kLog8Levels = 255;  // codes 1..255; code 0 = no depth

// code -> float32 metres (code 0 -> 0), FP64 values rounded to nearest
void log8_decode_table(float out[256]);

}  // namespace imloc
