// The float-field engine of the FFT phase-field-fracture library, compiled on its own so that the
// two precisions build in parallel.
#include "pff_engine.cuh"

namespace pffeng {
EngineBase *make_engine_f32(const rve_config &c) { return new Engine<float>(c); }
}  // namespace pffeng
