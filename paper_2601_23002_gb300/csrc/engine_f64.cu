// Plain FP64 engine: every step in double precision.
#include "engine_impl.cuh"

namespace ofdft {
template class Engine<double>;
IEngine* make_engine_f64(const CellSpec& c, int m_max) { return new Engine<double>(c, m_max); }
size_t engine_bytes(const CellSpec& c, int precision, int m_max) {
  if (precision == OFDFT_FP32) return Engine<float>(c, m_max).plan_bytes_estimate();
  return Engine<double>(c, m_max).plan_bytes_estimate();
}
}  // namespace ofdft
