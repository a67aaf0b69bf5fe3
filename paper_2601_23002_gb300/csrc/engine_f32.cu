// FP32-bulk engine: FFTs and pointwise terms in float, FP64 reductions,
// FP64 line search and setup tables.
#include "engine_impl.cuh"

namespace ofdft {
template class Engine<float>;
IEngine* make_engine_f32(const CellSpec& c, int m_max) { return new Engine<float>(c, m_max); }
}  // namespace ofdft
