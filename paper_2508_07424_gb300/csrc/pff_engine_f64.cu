// The double-field engine of the FFT phase-field-fracture library, compiled on its own so that the
// two precisions build in parallel.
#include "pff_engine.cuh"

namespace pffeng {
EngineBase *make_engine_f64(const rve_config &c) { return new Engine<double>(c); }
}  // namespace pffeng
